"""GPU benchmark expressions (Eqs. 9-21), fused ("Tensors") and per-component ("Arrays") forms, against
the oracle: bit for bit where the expression has no contraction (same roundings), and for the
"Arrays" form of the contractions (same summation order); the fused contractions (FMA, one factor at a
time) within 64 u of the sum of the absolute values of their terms."""
import numpy as np
import pytest

import gridgen
import oracle
from tests.parity import component_errors

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EQS = list(range(9, 22))


def run(eq, x, mode):
    import paper_1804_10120_gb300 as tl
    y = tl.tl_expr_eval(eq, torch.from_numpy(x).to(torch.device("cuda", 0)), mode=mode)
    torch.cuda.synchronize()
    return y.cpu().numpy()


@pytest.mark.parametrize("eq", EQS)
@pytest.mark.parametrize("n", [1, 300, 70001])
def test_expression_parity(eq, n):
    n_in, n_out = oracle.EXPR_ARITY[eq]
    x = gridgen.normal_fields(n_in, n, 100 + eq, 5000)
    ref = oracle.expr(eq, x)
    arrays = run(eq, x, "arrays")
    assert np.array_equal(arrays, ref), eq
    fused = run(eq, x, "fused")
    if eq in (18, 19, 20):
        # a-priori bound for a sum of products in a different order with FMA: |error| <= 64 u sum|terms|,
        # the sum of |terms| being the oracle on the absolute values of the inputs
        bound = 64 * 2.0 ** -53 * oracle.expr(eq, np.abs(x))
        assert np.all(np.abs(fused - ref) <= bound), eq
        assert component_errors(fused, ref).max() <= 1e-13
    else:
        assert np.array_equal(fused, ref), eq


def test_empty_and_arity():
    import paper_1804_10120_gb300 as tl
    for eq in EQS:
        assert tl.tl_expr_arity(eq) == oracle.EXPR_ARITY[eq]
    y = tl.tl_expr_eval(20, torch.empty((108, 0), dtype=torch.float64, device=torch.device("cuda", 0)))
    assert y.shape == (81, 0)
    with pytest.raises(tl.TLError):
        tl.tl_expr_arity(22)
