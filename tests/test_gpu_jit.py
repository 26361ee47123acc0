"""Kernels emitted by the runtime generator against the reference interpreter of the same programs,
and the generated metric-evolution chain against the chain oracle and the hand-written kernel."""
import numpy as np
import pytest

import gridgen
import oracle
from oracle.tensor_expr import Program
from tests.jit_programs import PROGRAMS
from tests.parity import TOL_F64, assert_components, component_errors

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def dev():
    return torch.device("cuda", 0)


@pytest.mark.parametrize("name", sorted(PROGRAMS))
@pytest.mark.parametrize("n", [1, 1000, 65537])
def test_generated_kernel_matches_interpreter(name, n):
    import paper_1804_10120_gb300 as tl
    k = tl.JitKernel(PROGRAMS[name])
    p = Program(PROGRAMS[name])
    if name.startswith("chain"):
        x = gridgen.random_grid(n, 71)
    else:
        x = gridgen.normal_fields(k.n_in, n, 71, 6000)
    y = k.launch(torch.from_numpy(x).to(dev()))
    torch.cuda.synchronize()
    y = y.cpu().numpy()
    ref = p.run(x)
    # generated code may contract a*b + c into an FMA: compare per component against the
    # component's scale (1e-12 for the chain, the 43-input program with a division)
    tol = TOL_F64 if name.startswith("chain") else 1e-13
    assert component_errors(y, ref).max() <= tol, name
    k.close()


def test_generated_chain_equals_chain_oracle_and_hand_kernel():
    import paper_1804_10120_gb300 as tl
    k = tl.JitKernel(PROGRAMS["chain"])
    x = gridgen.random_grid(1 << 20, 1)
    xd = torch.from_numpy(x).to(dev())
    y_gen = k.launch(xd)
    y_hand = tl.tl_dtg_forward(xd)
    torch.cuda.synchronize()
    idx = np.random.default_rng(0).integers(0, 1 << 20, 20000)
    ref = oracle.forward(np.ascontiguousarray(x[:, idx]))
    assert_components(y_gen[:, idx].cpu().numpy(), ref, TOL_F64, what="generated chain")
    assert component_errors(y_gen.cpu().numpy(), y_hand.cpu().numpy()).max() <= TOL_F64


def test_empty_launch_and_reuse_across_streams():
    import paper_1804_10120_gb300 as tl
    k = tl.JitKernel(PROGRAMS["eq21"])
    y = k.launch(torch.empty((10, 0), dtype=torch.float64, device=dev()))
    assert y.shape == (6, 0)
    x = torch.from_numpy(gridgen.normal_fields(10, 5000, 3, 6000)).to(dev())
    s = torch.cuda.Stream()
    y1 = k.launch(x)
    y2 = k.launch(x, stream=s)
    s.synchronize()
    torch.cuda.synchronize()
    assert torch.equal(y1, y2)



UNFUSED = [("statement", name) for name in sorted(PROGRAMS)] + \
          [("component", name) for name in ("chain", "eq14", "eq21", "listing17", "spatial_slice", "trace_div")]


@pytest.mark.parametrize("mode,name", UNFUSED)
def test_unfused_pipeline_matches_fused_and_interpreter(mode, name):
    """The program evaluated one kernel per assigned tensor or per stored component (intermediates
    through device memory, launched on a side stream) against the fused kernel and the reference
    interpreter."""
    from paper_1804_10120_gb300.statements import StatementPipeline
    n = 65537
    pl = StatementPipeline(PROGRAMS[name], mode)
    x = gridgen.random_grid(n, 72) if name.startswith("chain") else gridgen.normal_fields(pl.n_in, n, 72, 6000)
    xd = torch.from_numpy(x).to(dev())
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    y_st = pl.run(xd, stream=s)
    s.synchronize()
    y_fused = pl.fused.launch(xd)
    torch.cuda.synchronize()
    tol = TOL_F64 if name.startswith("chain") else 1e-13
    ref = Program(PROGRAMS[name]).run(x)
    assert component_errors(y_st.cpu().numpy(), ref).max() <= tol, name
    assert component_errors(y_st.cpu().numpy(), y_fused.cpu().numpy()).max() <= tol, name
    pl.close()


def test_generated_product_is_the_ieee_product():
    """A stand-alone product in a program becomes the generator's integer-pipe product: bit for bit
    the host CPU's IEEE product over the whole format (random bit patterns, both thresholds, ties)."""
    import paper_1804_10120_gb300 as tl
    from tests.test_gpu_f64_int import operands, same_bits
    k = tl.JitKernel("in a; in b; out c; c = a*b;")
    assert "tl_mul(" in k.source
    rng = np.random.default_rng(9)
    with np.errstate(all="ignore"):
        for a, b in operands(rng, 1 << 18):
            a, b = np.ascontiguousarray(a, np.float64), np.ascontiguousarray(b, np.float64)
            y = k.launch(torch.from_numpy(np.stack([a, b])).to(dev()))
            torch.cuda.synchronize()
            same_bits(y.cpu().numpy()[0], a * b)
    k.close()


def test_generated_chain_emits_fused_contractions():
    """The generated chain uses one integer-pipe product per contraction and FMAs for the rest (31
    stand-alone products, like the hand kernel), a Newton reciprocal for 1/det, and agrees with the
    hand kernel within the binary64 gate."""
    import paper_1804_10120_gb300 as tl
    from paper_1804_10120_gb300.programs import CHAIN
    k = tl.JitKernel(CHAIN)
    body = k.source[k.source.index("tl_jit_kernel"):]
    assert body.count("tl_mul(") == 31 and body.count("tl_rcp(") == 1 and " / " not in body
    xd = torch.from_numpy(gridgen.random_grid(100003, 5)).to(dev())
    y_gen = k.launch(xd)
    y_hand = tl.tl_dtg_forward(xd)
    torch.cuda.synchronize()
    assert component_errors(y_gen.cpu().numpy(), y_hand.cpu().numpy()).max() <= TOL_F64
    k.close()


def test_generated_chain_with_symmetric_footnote_sum():
    """With the footnote's sum written as a temporary symmetric in ij, the generator forms its 6 distinct
    values (one integer-pipe product and 2 FMAs each, then 9 subtractions: 21 FP64 operations) instead
    of 9 chains of 3 FMAs from d_j beta_i (27), as the hand kernel does: 6 more stand-alone products
    than the literal chain, the same outputs within the binary64 gate."""
    import paper_1804_10120_gb300 as tl
    from paper_1804_10120_gb300.programs import CHAIN_SYM
    k = tl.JitKernel(CHAIN_SYM)
    body = k.source[k.source.index("tl_jit_kernel"):]
    assert body.count("tl_mul(") == 31 + 6 and body.count("tl_rcp(") == 1
    x = gridgen.random_grid(100003, 6)
    xd = torch.from_numpy(x).to(dev())
    y_gen = k.launch(xd)
    y_hand = tl.tl_dtg_forward(xd)
    torch.cuda.synchronize()
    assert component_errors(y_gen.cpu().numpy(), y_hand.cpu().numpy()).max() <= TOL_F64
    idx = np.arange(0, 100003, 7)
    assert_components(y_gen.cpu().numpy()[:, idx], oracle.forward(np.ascontiguousarray(x[:, idx])), TOL_F64,
                      what="symmetric-sum chain")
    k.close()


def test_launch_bound_kept_after_loading():
    """The first launch checks the loaded kernel's local memory: the chain keeps three blocks per SM
    (80 registers, a few dozen bytes spilled), the rank-4 contraction stays at two, and both still
    match the reference interpreter."""
    import ctypes
    import paper_1804_10120_gb300 as tl
    from paper_1804_10120_gb300.programs import CHAIN_SYM
    from oracle.tensor_expr import Program
    L = tl.lib()
    L.tl_testing_jit_min_blocks.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32)]
    rank4 = "in B(3,3); in E(3,3,3,3); out A(3,3,3,3); A(i,j,k,l) = Sum(m, B(i,m)*E(m,j,k,l));"
    for text, want in ((CHAIN_SYM, 3), (rank4, 2)):
        k = tl.JitKernel(text)
        n = 1000
        x = gridgen.random_grid(n, 7) if text is CHAIN_SYM else gridgen.normal_fields(k.n_in, n, 7, 6000)
        y = k.launch(torch.from_numpy(x).to(dev()))
        torch.cuda.synchronize()
        b = ctypes.c_int32()
        assert L.tl_testing_jit_min_blocks(k._h, ctypes.byref(b)) == 0 and b.value == want
        ref = Program(text).run(x)
        assert component_errors(y.cpu().numpy(), ref).max() <= TOL_F64
        k.close()


def test_generated_chain_full_size():
    """The generated chain at the benchmark's size and launch (N = 2^24, seed 1, three blocks per SM):
    every point within the binary64 gate of the hand kernel, and a sample of points against the
    oracle."""
    import paper_1804_10120_gb300 as tl
    from paper_1804_10120_gb300.programs import CHAIN
    n = 1 << 24
    x = gridgen.random_grid(n, 1)
    xd = torch.from_numpy(x).to(dev())
    k = tl.JitKernel(CHAIN)
    y_gen = k.launch(xd)
    y_hand = tl.tl_dtg_forward(xd)
    torch.cuda.synchronize()
    err = ((y_gen - y_hand).abs().amax(dim=1) / y_hand.abs().amax(dim=1)).max().item()
    assert err <= TOL_F64, err
    rng = np.random.default_rng(13)
    idx = np.unique(np.concatenate([np.arange(256), np.arange(n - 256, n), rng.integers(0, n, 20000)]))
    yg = y_gen[:, torch.from_numpy(idx).to(dev())].cpu().numpy()
    assert_components(yg, oracle.forward(np.ascontiguousarray(x[:, idx])), TOL_F64, what="generated chain, N=2^24")
    del y_gen, y_hand, xd
    k.close()


@pytest.mark.parametrize("which", ["chain", "chain_sym"])
def test_generated_chain_conformal_grid_exact_zeros(which):
    """Conformally flat metric with beta = K = 0: the generated chain's nabla beta and d_t g vanish
    exactly, as the hand kernel's do, and Gamma matches the oracle."""
    import paper_1804_10120_gb300 as tl
    from paper_1804_10120_gb300.programs import CHAIN, CHAIN_SYM
    x = gridgen.conformal_grid(24)
    k = tl.JitKernel(CHAIN if which == "chain" else CHAIN_SYM)
    y = k.launch(torch.from_numpy(x).to(dev()))
    torch.cuda.synchronize()
    y = y.cpu().numpy()
    assert np.all(y[24:39] == 0.0)
    assert_components(y, oracle.forward(x), TOL_F64, what="generated %s, conformal" % which)
    k.close()
