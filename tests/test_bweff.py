"""Element counts of the effective-bandwidth metric (Sec. 5.1, Eq. 8) against the paper's worked
examples, and the count used for the fused chain."""
import os

from paper_1804_10120_gb300.bweff import Idx, Ref, count_elements, dtg_chain_refs, DTG_ELEMENTS

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "bw_eff_examples.txt")


def _gold():
    out = {}
    for line in open(GOLD):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            out[k] = int(v)
    return out


def test_paper_examples():
    g = _gold()
    a, b, c, i = Idx("a"), Idx("b"), Idx("c"), Idx("i")
    # C(Sym<0,1>, a, b) = Sum(c, A(a,c) * B(c,b)), spacetime indices
    refs = [Ref("C", (a, b), ((0, 1),)), Ref("A", (a, c)), Ref("B", (c, b))]
    assert count_elements(refs, {"a": 4, "b": 4, "c": 4}) == g["contraction_sym"]
    # D(Sym<0,1>, i, 0) = Sum(c, E(i+1, c) * F(c, 0))
    refs = [Ref("D", (i, 0), ((0, 1),)), Ref("E", (i + 1, c)), Ref("F", (c, 0))]
    assert count_elements(refs, {"i": 3, "c": 4}) == g["contraction_fixed_offset"]


def test_fused_chain_count():
    assert count_elements(dtg_chain_refs(), {"i": 3, "j": 3, "k": 3}) == DTG_ELEMENTS == 82


def test_adjoint_element_count():
    from paper_1804_10120_gb300.bweff import adjoint_elements
    assert adjoint_elements(24) == 34 + 24 + 43 == 101
