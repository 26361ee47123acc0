"""The runtime generator on the host: every program of the suite compiles through NVRTC (no device
needed), its component tables match the reference interpreter's, and programs that break the index
rules are rejected with a message."""
import pytest

from oracle.tensor_expr import Program
from tests.jit_programs import BAD, PROGRAMS


@pytest.fixture(scope="module")
def tl():
    from paper_1804_10120_gb300 import build
    build.build()
    import paper_1804_10120_gb300 as mod
    return mod


@pytest.mark.parametrize("name", sorted(PROGRAMS))
def test_compiles_with_matching_tables(tl, name):
    k = tl.JitKernel(PROGRAMS[name])
    p = Program(PROGRAMS[name])
    assert k.inputs == [(n, t) for n, t in p.inputs()]
    assert k.outputs == [(n, t) for n, t in p.outputs()]
    assert "tl_jit_kernel" in k.source and "__stcs" in k.source
    k.close()


@pytest.mark.parametrize("text", sorted(BAD))
def test_rejects_index_rule_violations(tl, text):
    with pytest.raises(tl.TLError) as ei:
        tl.JitKernel(text)
    assert BAD[text] in str(ei.value)


def test_chain_tables_match_the_fixed_abi(tl):
    """The chain program's tables coincide with tl_dtg_forward's 43 + 39 layout."""
    k = tl.JitKernel(PROGRAMS["chain"])
    assert k.n_in == 43 and k.n_out == 39
    assert k.inputs[6:9] == [("dg", (0, 0, 0)), ("dg", (0, 0, 1)), ("dg", (0, 0, 2))]
    assert k.inputs[30] == ("alpha", ())
    assert k.outputs[6 + 6 * 1 + 4] == ("Gamma", (1, 1, 2))
    assert k.outputs[24 + 3 * 2 + 1] == ("dbcov", (2, 1))



UNFUSED = [("statement", name) for name in sorted(PROGRAMS)] + \
          [("component", name) for name in ("chain", "eq14", "eq21", "listing17", "spatial_slice", "trace_div")]


@pytest.mark.parametrize("mode,name", UNFUSED)
def test_unfused_pipeline_routes_every_component(tl, mode, name):
    """Unfused stages: every component a stage loads is an input of the program or written by an
    earlier stage, and the stages together write every output of the fused kernel exactly once."""
    from paper_1804_10120_gb300.statements import StatementPipeline
    pl = StatementPipeline(PROGRAMS[name], mode)
    written = set(pl.fused.inputs)
    for k, keys in pl.stages:
        assert all(key in written for key, rd in zip(k.inputs, k.reads) if rd), name
        assert not (set(keys) & written), name
        written |= set(keys)
    assert set(pl.fused.outputs) <= written
    pl.close()


def test_unfused_pipelines_of_the_chain(tl):
    """Per tensor the chain splits into c, det, ginv, T, Gamma, dbcov, dtg with 25 temporary
    components (cofactors, determinant, bracket); per component it is 6+1+6+18+18+9+6 = 64 launches.
    Loaded plus stored elements per point: 82 fused, 171 per tensor, 331 per component (e.g. each
    Gamma component loads 3 ginv and 3 bracket components and stores 1)."""
    from paper_1804_10120_gb300.statements import StatementPipeline, split_components
    pl = StatementPipeline(PROGRAMS["chain"])
    assert [k.outputs[0][0] for k, _ in pl.stages] == ["c", "det", "ginv", "T", "Gamma", "dbcov", "dtg"]
    assert pl.intermediate_components() == 6 + 1 + 18
    assert pl.fused.n_in + pl.fused.n_out == 82
    assert pl.elements_per_point() == 171
    pl.close()
    pieces = split_components(PROGRAMS["chain"])
    assert len(pieces) == 64
    assert [key for key, _ in pieces].count(("Gamma", (2, 1, 2))) == 1
    assert ("Gamma", (2, 2, 1)) not in [key for key, _ in pieces]
    g212 = dict(pieces)[("Gamma", (2, 1, 2))]
    assert "Sum(l, ginv(2,l)*T(l,1,2))" in g212
    pl = StatementPipeline(PROGRAMS["chain"], "component")
    assert pl.launches == 64 and pl.intermediate_components() == 25
    assert pl.elements_per_point() == 331
    pl.close()


def test_component_split_of_fixed_and_offset_indices():
    """listing17's D(i,0) = Sum(c, E(i+1,c) F(c,0)) over i < 3: the offset is resolved per component
    and the fixed-index statements that follow keep their own components."""
    from paper_1804_10120_gb300.statements import split_components
    pieces = dict(split_components(PROGRAMS["listing17"]))
    assert "Sum(c, E(3,c)*F(c,0))" in pieces[("D", (0, 2))]
    assert "E(0,0)" in pieces[("D", (0, 3))]
    assert len(pieces) == 10


def test_launch_bound_follows_the_spill_report(tl):
    """A program whose kernel fits three 256-thread blocks per SM without spilling more than 128 bytes is
    built for three (the chain); one that would spill more is rebuilt for two (a rank-4 contraction
    holding its 81 results); and the generated kernel stores each output right after the statement
    that finishes it and loads each input just before its first use."""
    import ctypes
    from paper_1804_10120_gb300.programs import CHAIN, CHAIN_SYM
    L = tl.lib()
    L.tl_testing_jit_min_blocks.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32)]
    L.tl_testing_jit_min_blocks.restype = ctypes.c_int

    def blocks(text):
        k = tl.JitKernel(text)
        b = ctypes.c_int32()
        assert L.tl_testing_jit_min_blocks(k._h, ctypes.byref(b)) == 0
        src = k.source
        k.close()
        return b.value, src

    b_chain, src = blocks(CHAIN_SYM)
    assert b_chain == 3 and blocks(CHAIN)[0] == 3
    assert blocks("in B(3,3); in E(3,3,3,3); out A(3,3,3,3); A(i,j,k,l) = Sum(m, B(i,m)*E(m,j,k,l));")[0] == 2
    body = src[src.index("tl_jit_kernel("):]
    # Gamma (out[6..23]) is stored before beta (in[31]) is loaded; K (in[24]) is loaded after dbcov is stored
    assert body.index("a.out[6] + x") < body.index("__ldcs(a.in[31] + x)") < body.index("a.out[24] + x")
    assert body.index("a.out[32] + x") < body.index("__ldcs(a.in[24] + x)")
    assert body.index('"l"(a.in[24] + x)') < body.index("__ldcs(a.in[0] + x)")   # prefetched at the top
    assert L.tl_testing_jit_min_blocks(None, ctypes.byref(ctypes.c_int32())) == 1
