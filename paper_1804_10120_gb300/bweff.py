"""Effective-bandwidth accounting (Sec. 5.1, Eq. 8 of Lewis & Pfeiffer, arXiv:1804.10120).

BW_eff = 8 bytes * (N_e * N + N_d) / t, where N is the number of grid points, N_e the number of distinct
stored tensor elements an operation reads or writes, and N_d the number of doubles outside grid arrays.
Each distinct element is one grid-length array that must cross HBM once, whatever the kernel does
internally.  This module counts N_e for index expressions with symmetric slots, fixed indices and
index offsets, and holds the counts of the fused metric-evolution chain.
"""
import itertools
from dataclasses import dataclass, field
from typing import Dict, Sequence, Tuple, Union


@dataclass(frozen=True)
class Idx:
    """A symbolic index letter, optionally shifted by a constant offset (e.g. i+1)."""
    name: str
    offset: int = 0

    def __add__(self, k):
        return Idx(self.name, self.offset + k)


Slot = Union[Idx, int]


@dataclass(frozen=True)
class Ref:
    """One tensor reference in an expression: name, one entry per index slot, and the groups of slots
    that are symmetric (stored once per unordered tuple)."""
    name: str
    slots: Tuple[Slot, ...]
    sym: Tuple[Tuple[int, ...], ...] = field(default=())


def _storage_key(ref: Ref, values: Tuple[int, ...]):
    v = list(values)
    for group in ref.sym:
        sorted_vals = sorted(v[s] for s in group)
        for s, val in zip(sorted(group), sorted_vals):
            v[s] = val
    return (ref.name, tuple(v))


def count_elements(refs: Sequence[Ref], dims: Dict[str, int]) -> int:
    """N_e: the number of distinct stored elements touched by the references, with every index
    letter running over range(dims[letter])."""
    letters = sorted({s.name for r in refs for s in r.slots if isinstance(s, Idx)})
    keys = set()
    for assign in itertools.product(*[range(dims[l]) for l in letters]):
        env = dict(zip(letters, assign))
        for r in refs:
            vals = tuple(env[s.name] + s.offset if isinstance(s, Idx) else s for s in r.slots)
            keys.add(_storage_key(r, vals))
    return len(keys)


def dtg_chain_refs():
    """The stored elements of the fused chain: inputs g_ij, d_k g_ij, K_ij, alpha, beta_i, d_j beta_i;
    outputs g^ij, Gamma^i_jk, nabla_j beta_i, d_t g_ij (Eqs. 2-3 and the footnote to Listing 1)."""
    i, j, k = Idx("i"), Idx("j"), Idx("k")
    return [
        Ref("g", (i, j), ((0, 1),)),
        Ref("dg", (i, j, k), ((0, 1),)),
        Ref("K", (i, j), ((0, 1),)),
        Ref("alpha", ()),
        Ref("beta", (i,)),
        Ref("dbeta", (i, j)),
        Ref("ginv", (i, j), ((0, 1),)),
        Ref("Gamma", (i, j, k), ((1, 2),)),
        Ref("dbcov", (i, j)),
        Ref("dtg", (i, j), ((0, 1),)),
    ]


# Elements read and written by one pass of the fused forward chain.
DTG_IN_ELEMENTS = 43
DTG_OUT_ELEMENTS = 39
DTG_ELEMENTS = DTG_IN_ELEMENTS + DTG_OUT_ELEMENTS
# Adjoint alone: the inputs it reads (all but the 9 d_j beta_i, on which the gradient does not depend),
# the upstream gradients actually read and the 43 input gradients written.
ADJOINT_IN_ELEMENTS = DTG_IN_ELEMENTS - 9


def adjoint_elements(n_upstream: int) -> int:
    return ADJOINT_IN_ELEMENTS + n_upstream + DTG_IN_ELEMENTS


def bytes_per_point(elements: int, word: int = 8) -> int:
    return elements * word
