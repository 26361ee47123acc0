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
