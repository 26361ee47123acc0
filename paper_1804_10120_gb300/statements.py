"""A tensor-index program evaluated unfused, the way the paper measures its "Arrays" baseline and the
evaluation model of its expression-template library (Secs. 3-5): one kernel per assigned tensor
(mode "statement") or one kernel per stored component (mode "component"), every intermediate stored
to and re-read from device memory.  The fused program (one kernel for all statements) is the design
this package uses; all three are built by the same runtime generator, so comparing them isolates
what fusion saves."""
import itertools
import re

_DECL = re.compile(r"^(in|out|temp)\s+(\w+)")
_TENSOR = re.compile(r"^(\w+)\s*(?:\(([^)]*)\))?\s*(.*)$")


def _items(text):
    text = re.sub(r"(#|//)[^\n]*", "", text)
    return [t.strip() for t in text.split(";") if t.strip()]


def _parse(text):
    """decls: name -> (kind, declaration text, dims, sym pairs); index ranges; statements (lhs, rhs)."""
    decls, ranges, stmts = {}, {}, []
    for it in _items(text):
        m = _DECL.match(it)
        if m:
            body = it[m.end(1):].strip()
            t = _TENSOR.match(body)
            dims = tuple(int(v) for v in t.group(2).split(",")) if t.group(2) else ()
            syms = [tuple(int(v) for v in p) for p in re.findall(r"sym\s*\(\s*(\d+)\s*,\s*(\d+)\s*\)", t.group(3))]
            decls[m.group(2)] = (m.group(1), body, dims, syms)
        elif it.startswith("index"):
            for letter, r in re.findall(r"\b([a-z])\s*\(\s*(\d+)\s*\)", it[5:]):
                ranges[letter] = int(r)
        else:
            lhs, rhs = it.split("=", 1)
            stmts.append((lhs.strip(), rhs.strip()))
    return decls, ranges, stmts


def _reads(rhs, decls, own):
    out = []
    for r in re.findall(r"\b([A-Za-z_]\w*)\b", rhs):
        if r in decls and r != own and r not in out:
            out.append(r)
    return out


def split_program(text):
    """Per assigned tensor, in order of first assignment: the program that computes it alone, as
    [(tensor name, program text)].  Every tensor a piece reads is an `in` of that piece and the
    assigned tensor its only `out`; `index` declarations are copied to every piece.  Statements that
    assign parts of one tensor (fixed-index left-hand sides) stay together in one piece."""
    decls, ranges, stmts = _parse(text)
    index_line = ["index " + ", ".join("%s(%d)" % kv for kv in sorted(ranges.items())) + ";"] if ranges else []
    groups = {}
    for lhs, rhs in stmts:
        name = re.match(r"(\w+)", lhs).group(1)
        g = groups.setdefault(name, ([], []))
        g[0].append("%s = %s;" % (lhs, rhs))
        g[1].extend(r for r in _reads(rhs, decls, name) if r not in g[1])
    return [(name, "\n".join(index_line + ["in %s;" % decls[r][1] for r in reads] + ["out %s;" % decls[name][1]]
                             + sts)) for name, (sts, reads) in groups.items()]


def _canonical(tup, syms):
    t = list(tup)
    for a, b in syms:
        if t[a] > t[b]:
            t[a], t[b] = t[b], t[a]
    return tuple(t)


def _substitute(rhs, values):
    """rhs with every free letter (and letter+c, letter-c) of `values` replaced by its integer value."""
    if not values:
        return rhs
    pat = re.compile(r"\b([%s])\b(\s*[+-]\s*\d+)?(?!\s*\()" % "".join(values))

    def rep(m):
        v = values[m.group(1)]
        if m.group(2):
            v += int(m.group(2).replace(" ", ""))
        return str(v)
    return pat.sub(rep, rhs)


def split_components(text):
    """Per stored component of every assigned tensor, in statement order: the program that computes
    that component alone, as [((tensor name, index tuple), program text)].  A statement computes the
    stored components its left-hand side reaches first (row-major over its free letters, symmetric
    pairs folded onto ascending indices); its right-hand side is evaluated with the free letters
    fixed to that reach.  The piece writes one scalar `out`; every tensor it reads is a whole `in`."""
    decls, ranges, stmts = _parse(text)
    done, pieces = set(), []
    for lhs, rhs in stmts:
        m = re.match(r"(\w+)\s*(?:\(([^)]*)\))?", lhs)
        name = m.group(1)
        dims, syms = decls[name][2], decls[name][3]
        slots = [s.strip() for s in m.group(2).split(",")] if m.group(2) else []
        letters = list(dict.fromkeys(s for s in slots if s.isalpha()))
        for letter in letters:
            if letter in decls:
                raise ValueError("free letter %r is also a tensor name" % letter)
        span = [ranges.get(l, dims[slots.index(l)]) for l in letters]
        sum_letters = set(re.findall(r"Sum\s*\(\s*([a-z])\s*,", rhs))
        idx_lines = ["index " + ", ".join("%s(%d)" % (l, ranges[l]) for l in sorted(sum_letters) if l in ranges) + ";"] \
            if any(l in ranges for l in sum_letters) else []
        reads = _reads(rhs, decls, name)
        for vals in itertools.product(*[range(r) for r in span]):
            values = dict(zip(letters, vals))
            tup = _canonical(tuple(values[s] if s.isalpha() else int(s) for s in slots), syms)
            if (name, tup) in done:
                continue
            done.add((name, tup))
            scalar = "%s__%s" % (name, "_".join(map(str, tup))) if tup else name + "__"
            body = idx_lines + ["in %s;" % decls[r][1] for r in reads] + ["out %s;" % scalar,
                                                                          "%s = %s;" % (scalar, _substitute(rhs, values))]
            pieces.append(((name, tup), "\n".join(body)))
    return pieces


class StatementPipeline:
    """`text` compiled by the generator as one fused kernel (`fused`) and as unfused `stages`: one
    kernel per assigned tensor (mode "statement") or per stored component (mode "component").  `run`
    evaluates the stages in order with the fused kernel's input and output component tables."""

    def __init__(self, text, mode="statement"):
        from . import JitKernel
        if mode not in ("statement", "component"):
            raise ValueError("mode must be 'statement' or 'component'")
        self.mode = mode
        self.fused = JitKernel(text)
        self.n_in, self.n_out = self.fused.n_in, self.fused.n_out
        out_row = {key: r for r, key in enumerate(self.fused.outputs)}
        # where every component lives: ("in", row), ("out", row) or ("temp", row)
        self._loc = {key: ("in", r) for r, key in enumerate(self.fused.inputs)}
        self.stages = []     # (kernel, [component written by each output entry])
        self.n_temp = 0
        if mode == "statement":
            for _, prog in split_program(text):
                k = JitKernel(prog)
                self.stages.append((k, list(k.outputs)))
        else:
            for key, prog in split_components(text):
                self.stages.append((JitKernel(prog), [key]))
        for _, keys in self.stages:
            for key in keys:
                if key in out_row:
                    self._loc[key] = ("out", out_row[key])
                else:
                    self._loc[key] = ("temp", self.n_temp)
                    self.n_temp += 1

    @property
    def launches(self):
        return len(self.stages)

    def intermediate_components(self):
        """Components stored to device memory between stages and read back (temporaries only)."""
        return self.n_temp

    def elements_per_point(self):
        """Array elements every stage loads or stores, summed: the unfused form's algorithmic traffic
        per point in units of one element (the fused kernel's is n_in + n_out)."""
        return sum(sum(k.reads) + k.n_out for k, _ in self.stages)

    def run(self, inputs, outputs=None, stream=None):
        """inputs: [n_in, n] device float64 (or n_in rows) in the fused kernel's input order.  Returns
        [n_out, n] in its output order."""
        import torch
        from . import _rows
        rows_in = _rows(inputs, self.n_in, "inputs")
        n, dev = rows_in[0].shape[0], rows_in[0].device
        if outputs is None:
            outputs = torch.empty((self.n_out, n), dtype=torch.float64, device=dev)
        bufs = {"in": rows_in, "out": _rows(outputs, self.n_out, "outputs"), "temp": []}
        if self.n_temp:
            t = torch.empty((self.n_temp, n), dtype=torch.float64, device=dev)
            if stream is not None and hasattr(stream, "cuda_stream"):
                t.record_stream(stream)     # freed after this call; in use until `stream` gets there
            bufs["temp"] = list(t)
        for k, keys in self.stages:
            # entries the kernel does not load still need a valid array: any program input serves
            src = [bufs[self._loc[key][0]][self._loc[key][1]] if rd else rows_in[0]
                   for key, rd in zip(k.inputs, k.reads)]
            dst = [bufs[self._loc[key][0]][self._loc[key][1]] for key in keys]
            k.launch(src, dst, stream=stream)
        return outputs

    def close(self):
        self.fused.close()
        for k, _ in self.stages:
            k.close()
