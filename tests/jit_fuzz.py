"""Seeded random tensor-index programs for the generator tests (valid by construction: every + / -
joins terms with the same free letters, every repeated letter is bound by a Sum)."""
import random

LETTERS = "ijklmnopq"


def _term(rng, free, fresh, depth, inputs):
    """An expression whose free letters are exactly `free` (a tuple)."""
    choice = rng.random()
    if len(free) > 3:                      # no input has rank > 3: split the letters over a product
        k = len(free) // 2
        return "%s*%s" % (_term(rng, tuple(free[:k]), fresh, depth - 1, inputs),
                          _term(rng, tuple(free[k:]), fresh, depth - 1, inputs))
    if depth <= 0 or choice < 0.35:
        rank = len(free)
        # an input of rank >= |free|; extra slots get fixed indices
        cands = [(name, r, sym) for name, r, sym in inputs if r >= rank]
        name, r, sym = rng.choice(cands)
        slots = list(range(r))
        rng.shuffle(slots)
        idx = [str(rng.randrange(3))] * r
        for letter, s in zip(free, slots[:rank]):
            idx[s] = letter
        ref = "%s(%s)" % (name, ",".join(idx)) if r else name
        return ref
    if choice < 0.6 and len(free) >= 1:
        # product: split the free letters between the two factors
        k = rng.randrange(len(free) + 1)
        f1, f2 = tuple(free[:k]), tuple(free[k:])
        return "%s*%s" % (_term(rng, f1, fresh, depth - 1, inputs), _term(rng, f2, fresh, depth - 1, inputs))
    if choice < 0.8 and fresh and len(free) < 3:
        letter = fresh[0]
        body = _term(rng, tuple(free) + (letter,), fresh[1:], depth - 1, inputs)
        # the Sum's letter appears in the operand at least once by construction
        return "Sum(%s, %s)" % (letter, body)
    if choice < 0.9:
        return "%s*%s" % (rng.choice(["0.5", "2", "-3", "1.25", "0.1"]), _term(rng, free, fresh, depth - 1, inputs))
    return "(%s)" % _expr(rng, free, fresh, depth - 1, inputs)


def _expr(rng, free, fresh, depth, inputs):
    terms = [_term(rng, free, fresh, depth, inputs) for _ in range(rng.randrange(1, 4))]
    out = terms[0]
    for t in terms[1:]:
        out += rng.choice([" + ", " - "]) + t
    return out


def random_program(seed):
    rng = random.Random(seed)
    inputs = [("a", 0, False), ("v", 1, False), ("w", 1, False), ("M", 2, rng.random() < 0.5), ("N", 2, False),
              ("R", 3, rng.random() < 0.5)]
    decl = []
    for name, r, sym in inputs:
        dims = "(%s)" % ",".join(["3"] * r) if r else ""
        decl.append("in %s%s%s;" % (name, dims, " sym(0,1)" if sym else ""))
    stmts = []
    for o in range(rng.randrange(1, 3)):
        rank = rng.randrange(0, 3)
        free = tuple(LETTERS[:rank])
        fresh = LETTERS[rank:rank + 3]
        sym = rank == 2 and rng.random() < 0.4
        name = "O%d" % o
        decl.append("out %s%s%s;" % (name, "(%s)" % ",".join(["3"] * rank) if rank else "", " sym(0,1)" if sym else ""))
        lhs = "%s(%s)" % (name, ",".join(free)) if rank else name
        stmts.append("%s = %s;" % (lhs, _expr(rng, free, fresh, 3, inputs)))
    return "\n".join(decl + stmts)
