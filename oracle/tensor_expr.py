"""Reference interpreter for tensor-index programs (test infrastructure only).

An independent, slow evaluator of the program language accepted by the runtime generator: declarations
`in|out|temp NAME(d0,...) sym(a,b)...;`, statements `NAME(idx,...) = EXPR;` with index letters, offsets
(i+1, i-1), fixed integers, + - * / (division by scalars), unary minus, parentheses and Sum(l, EXPR).
`index l(d);` gives a letter a range other than its slot's dimension.  Each stored component a
statement's left-hand side reaches is evaluated once, at the first index assignment (row-major) that
reaches it, term by term over numpy arrays of grid values, with explicit Python loops over index
values; sums and products are taken left to right as written.  It follows the index-notation semantics
of the paper's expressions (Sec. 1, Eqs. 5-6; Sec. 2) and shares no code with the CUDA library.
"""
import itertools
import re

import numpy as np

_TOKEN = re.compile(r"\s*(?:(#[^\n]*|//[^\n]*)|(\d+\.\d*(?:[eE][-+]?\d+)?|\.\d+(?:[eE][-+]?\d+)?|\d+(?:[eE][-+]?\d+)?)|([A-Za-z_]\w*)|(.))")


def _tokens(text):
    out = []
    for m in _TOKEN.finditer(text):
        if m.group(1):
            continue
        if m.group(2):
            out.append(("num", m.group(2)))
        elif m.group(3):
            out.append(("id", m.group(3)))
        elif m.group(4) and not m.group(4).isspace():
            out.append(("op", m.group(4)))
    return out


class Decl:
    def __init__(self, kind, name, dims, sym):
        self.kind, self.name, self.dims, self.sym = kind, name, dims, sym

    def canonical(self, tup):
        t = list(tup)
        changed = True
        while changed:
            changed = False
            for a, b in self.sym:
                if t[a] > t[b]:
                    t[a], t[b] = t[b], t[a]
                    changed = True
        return tuple(t)

    def stored(self):
        return [t for t in itertools.product(*[range(d) for d in self.dims]) if self.canonical(t) == t]


class Program:
    def __init__(self, text):
        self.toks = _tokens(text)
        self.pos = 0
        self.decls = {}
        self.ranges = {}
        self.order = []
        self.stmts = []
        while self.pos < len(self.toks):
            kind, val = self.toks[self.pos]
            nxt = self.toks[self.pos + 1] if self.pos + 1 < len(self.toks) else ("", "")
            if kind == "id" and val == "index" and nxt[0] == "id":
                self.pos += 1
                while True:
                    letter = self._take()[1]
                    self._take("(")
                    self.ranges[letter] = int(self._take()[1])
                    self._take(")")
                    if self._peek()[1] != ",":
                        break
                    self._take(",")
                self._take(";")
            elif kind == "id" and val in ("in", "out", "temp") and nxt[0] == "id":
                self.pos += 1
                self._decl(val)
            else:
                self._stmt()

    # -- parsing
    def _peek(self):
        return self.toks[self.pos] if self.pos < len(self.toks) else ("eof", "")

    def _take(self, val=None):
        tok = self._peek()
        if val is not None and tok[1] != val:
            raise SyntaxError("expected %r, found %r" % (val, tok[1]))
        self.pos += 1
        return tok

    def _decl(self, kind):
        name = self._take()[1]
        dims = []
        if self._peek()[1] == "(":
            self._take("(")
            while self._peek()[1] != ")":
                dims.append(int(self._take()[1]))
                if self._peek()[1] == ",":
                    self._take(",")
            self._take(")")
        sym = []
        while self._peek()[1] == "sym":
            self._take("sym")
            self._take("(")
            a = int(self._take()[1])
            self._take(",")
            b = int(self._take()[1])
            self._take(")")
            sym.append((min(a, b), max(a, b)))
        self._take(";")
        self.decls[name] = Decl(kind, name, dims, sym)
        self.order.append(name)

    def _indices(self):
        idx = []
        if self._peek()[1] != "(":
            return idx
        self._take("(")
        while self._peek()[1] != ")":
            kind, val = self._take()
            if kind == "num":
                idx.append(("fixed", int(val)))
            else:
                off = 0
                if self._peek()[1] in "+-" and self._peek()[1] != "" and self.toks[self.pos + 1][0] == "num":
                    sign = 1 if self._take()[1] == "+" else -1
                    off = sign * int(self._take()[1])
                idx.append(("letter", val, off))
            if self._peek()[1] == ",":
                self._take(",")
        self._take(")")
        return idx

    def _stmt(self):
        name = self._take()[1]
        lhs = self._indices()
        self._take("=")
        rhs = self._sum()
        self._take(";")
        self.stmts.append((name, lhs, rhs))

    def _sum(self):
        node = self._prod()
        while self._peek()[1] in ("+", "-"):
            op = self._take()[1]
            node = (op, node, self._prod())
        return node

    def _prod(self):
        node = self._unary()
        while self._peek()[1] in ("*", "/"):
            op = self._take()[1]
            node = (op, node, self._unary())
        return node

    def _unary(self):
        if self._peek()[1] == "-":
            self._take("-")
            return ("neg", self._unary())
        if self._peek()[1] == "(":
            self._take("(")
            node = self._sum()
            self._take(")")
            return node
        kind, val = self._take()
        if kind == "num":
            return ("num", float(val))
        if val == "Sum":
            self._take("(")
            letter = self._take()[1]
            self._take(",")
            body = self._sum()
            self._take(")")
            return ("Sum", letter, body)
        return ("ref", val, self._indices())

    # -- evaluation
    def _dim_of(self, node, letter):
        if node[0] == "ref":
            decl = self.decls[node[1]]
            for s, ix in enumerate(node[2]):
                if ix[0] == "letter" and ix[1] == letter:
                    return self.ranges.get(letter, decl.dims[s])
            return None
        for child in node[1:]:
            if isinstance(child, tuple):
                d = self._dim_of(child, letter)
                if d is not None:
                    return d
        return None

    def _eval(self, node, env, values):
        op = node[0]
        if op == "num":
            return node[1]
        if op == "ref":
            decl = self.decls[node[1]]
            tup = tuple(ix[1] if ix[0] == "fixed" else env[ix[1]] + ix[2] for ix in node[2])
            for v, d in zip(tup, decl.dims):
                if not 0 <= v < d:
                    raise IndexError("index out of range for %s" % node[1])
            return values[node[1]][decl.canonical(tup)]
        if op == "neg":
            return -self._eval(node[1], env, values)
        if op == "Sum":
            letter = node[1]
            total = None
            for v in range(self._dim_of(node[2], letter)):
                term = self._eval(node[2], dict(env, **{letter: v}), values)
                total = term if total is None else total + term
            return total
        a = self._eval(node[1], env, values)
        b = self._eval(node[2], env, values)
        return {"+": lambda: a + b, "-": lambda: a - b, "*": lambda: a * b, "/": lambda: a / b}[op]()

    def inputs(self):
        return [(n, t) for n in self.order if self.decls[n].kind == "in" for t in self.decls[n].stored()]

    def outputs(self):
        return [(n, t) for n in self.order if self.decls[n].kind == "out" for t in self.decls[n].stored()]

    def run(self, inputs):
        """inputs: [n_in, n] array in the table order of inputs(); returns [n_out, n]."""
        table = self.inputs()
        assert len(inputs) == len(table)
        values = {n: {} for n in self.order}
        for (name, tup), arr in zip(table, inputs):
            values[name][tup] = np.asarray(arr, dtype=np.float64)
        for name, lhs, rhs in self.stmts:
            decl = self.decls[name]
            letters = []
            for ix in lhs:
                if ix[0] == "letter" and ix[1] not in letters:
                    letters.append(ix[1])
            dims = {ix[1]: self.ranges.get(ix[1], decl.dims[s]) for s, ix in enumerate(lhs) if ix[0] == "letter"}
            new = {}
            for combo in itertools.product(*[range(dims[l]) for l in letters]):
                env = dict(zip(letters, combo))
                tup = decl.canonical(tuple(ix[1] if ix[0] == "fixed" else env[ix[1]] for ix in lhs))
                if tup not in new:          # first assignment reaching this stored element
                    new[tup] = self._eval(rhs, env, values)
            values[name].update(new)
        n = np.asarray(inputs[0]).shape[-1] if len(inputs) else 0
        return np.stack([np.broadcast_to(np.asarray(values[name][tup], dtype=np.float64), (n,))
                         for name, tup in self.outputs()])
