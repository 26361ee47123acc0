"""Randomised programs: the generator and the reference interpreter agree on the component tables
(host, through NVRTC) and, on the GPU, on every output."""
import numpy as np
import pytest

import gridgen
from oracle.tensor_expr import Program
from tests.jit_fuzz import random_program
from tests.parity import component_errors

SEEDS = list(range(40))


@pytest.fixture(scope="module")
def tl():
    from paper_1804_10120_gb300 import build
    build.build()
    import paper_1804_10120_gb300 as mod
    return mod


@pytest.mark.parametrize("seed", SEEDS)
def test_random_program_tables(tl, seed):
    text = random_program(seed)
    k = tl.JitKernel(text)
    p = Program(text)
    assert k.inputs == list(p.inputs()) and k.outputs == list(p.outputs()), text
    k.close()


@pytest.mark.gpu
@pytest.mark.parametrize("seed", SEEDS)
def test_random_program_values(tl, seed):
    import torch
    text = random_program(seed)
    k = tl.JitKernel(text)
    p = Program(text)
    n = 777
    x = gridgen.normal_fields(k.n_in, n, 900 + seed, 7000)
    y = k.launch(torch.from_numpy(x).to(torch.device("cuda", 0)))
    torch.cuda.synchronize()
    ref = p.run(x)
    # a-priori bound: the same terms, possibly in another order, with FMA contraction and exact
    # cancellation of equal addends: |error| <= 64 u * (the interpreter on |inputs| with every - as +)
    absref = Program(text.replace(" - ", " + ").replace("-3", "3")).run(np.abs(x))
    assert np.all(np.abs(y.cpu().numpy() - ref) <= 64 * 2.0 ** -53 * absref + 1e-300), text
    k.close()
