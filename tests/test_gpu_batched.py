"""Batched multi-grid forward (one persistent launch over many uneven subgrids) against the oracle and
bit for bit against the single-grid kernel, in and out of a CUDA graph, before and after tuning."""
import numpy as np
import pytest

import gridgen
import oracle
from tests.parity import TOL_F64, assert_components

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def dev():
    return torch.device("cuda", 0)


def make_batch(sides, seed, dtype=torch.float64):
    """One grid per side (n = side^3), grid d drawing from its own streams (base 64 d)."""
    xs, ys, hosts = [], [], []
    for d, side in enumerate(sides):
        n = side ** 3
        x = gridgen.random_grid(n, seed, stream_base=gridgen.STREAMS_PER_FIELD * d)
        hosts.append(x)
        xs.append(torch.from_numpy(x).to(dev(), dtype))
        ys.append(torch.full((39, n), float("nan"), dtype=dtype, device=dev()))
    return hosts, xs, ys


@pytest.mark.parametrize("dtype", ["f64", "f64_ff"])
def test_small_batch_matches_oracle_and_single_grid(dtype):
    import paper_1804_10120_gb300 as tl
    sides = [8, 3, 12, 1, 9, 16, 5, 0, 10]
    hosts, xs, ys = make_batch(sides, 21)
    plan = tl.tl_dtg_batched_prepare(xs, ys, dtype=dtype)
    plan.launch()
    plan.check()
    for x, xd, y in zip(hosts, xs, ys):
        yb = y.cpu().numpy()
        assert_components(yb, oracle.forward(x), TOL_F64, what="batched %s" % dtype)
        ys_single = tl.tl_dtg_forward(xd, dtype=dtype)
        torch.cuda.synchronize()
        assert np.array_equal(ys_single.cpu().numpy(), yb)   # same per-point code: bitwise
    plan.close()


def test_every_config_and_graph_capture():
    import paper_1804_10120_gb300 as tl
    sides = [int(s) for s in np.random.default_rng(5).integers(2, 20, 40)]
    hosts, xs, ys = make_batch(sides, 22)
    plan = tl.BatchPlan(xs, ys)
    refs = [tl.tl_dtg_forward(x) for x in xs]
    torch.cuda.synchronize()
    for threads in (128, 256, 512):
        for bps in (1, 2):
            for ppt in (1, 2, 4):
                for y in ys:
                    y.fill_(float("nan"))
                try:
                    plan.set_config(threads, bps, ppt)
                except tl.TLError as e:          # beyond this kernel's occupancy
                    assert e.status == 1
                    continue
                assert plan.points_per_thread == ppt
                plan.launch()
                torch.cuda.synchronize()
                for y, r in zip(ys, refs):
                    assert torch.equal(y, r), (threads, bps, ppt)
    with pytest.raises(tl.TLError):
        plan.set_config(256, 1, 3)
    # CUDA graph: capture one launch, replay twice
    for y in ys:
        y.fill_(float("nan"))
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        plan.launch(stream=s)
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    for y, r in zip(ys, refs):
        assert torch.equal(y, r)
    plan.check()


def test_tuner_picks_a_valid_config(tmp_path, monkeypatch):
    import paper_1804_10120_gb300 as tl
    monkeypatch.setenv("TL_TUNE_CACHE", str(tmp_path / "tune.txt"))
    sides = [16, 20, 24, 12]
    hosts, xs, ys = make_batch(sides, 23)
    plan = tl.BatchPlan(xs, ys)
    t, b = plan.tune()
    q = plan.points_per_thread
    assert t in (128, 256, 512) and b >= 1 and q in (1, 2, 4)
    text = (tmp_path / "tune.txt").read_text()
    assert "batched" in text and ("%d %d %d" % (t, b, q)) in text
    st = plan.staging
    assert st in (0, 2, 3) and (st == 0 or q == 1)
    assert ("%d %d %d %d" % (t, b, q, st)) in text
    plan2 = tl.BatchPlan(xs, ys)             # same shape: configuration from the cache
    assert plan2.config == (t, b) and plan2.points_per_thread == q and plan2.staging == st
    plan2.launch()
    torch.cuda.synchronize()
    for x, y in zip(hosts, ys):
        assert_components(y.cpu().numpy(), oracle.forward(x), TOL_F64, what="tuned")


def test_multi_domain_600_grids_sampled():
    """600 subgrids, side ~ U{8..48} (seed 2): parity on a sample of grids, bitwise equality with the
    single-grid kernel on every grid."""
    import paper_1804_10120_gb300 as tl
    sides = gridgen.subgrid_sides(600, 2)
    assert min(sides) >= 8 and max(sides) <= 48
    hosts, xs, ys = make_batch(sides, 2)
    plan = tl.BatchPlan(xs, ys)
    plan.launch()
    torch.cuda.synchronize()
    plan.check()
    for d in range(0, 600, 37):
        assert_components(ys[d].cpu().numpy(), oracle.forward(hosts[d]), TOL_F64, what="grid %d" % d)
    for x, y in zip(xs, ys):
        assert torch.equal(tl.tl_dtg_forward(x), y)


def test_empty_batch():
    import paper_1804_10120_gb300 as tl
    plan = tl.BatchPlan([], [])
    plan.launch()
    plan.check()
    x = torch.empty((43, 0), dtype=torch.float64, device=dev())
    y = torch.empty((39, 0), dtype=torch.float64, device=dev())
    plan = tl.BatchPlan([x], [y])
    plan.launch()
    plan.check()


def test_f32_batch():
    import paper_1804_10120_gb300 as tl
    sides = [7, 13, 4]
    hosts, xs, ys = make_batch(sides, 24, dtype=torch.float32)
    plan = tl.BatchPlan(xs, ys, dtype="f32")
    plan.launch()
    for x, y in zip(xs, ys):
        assert torch.equal(tl.tl_dtg_forward(x, dtype="f32"), y)


@pytest.mark.parametrize("dtype", ["f64", "f64_ff", "f32"])
def test_array_and_scattered_row_tables(dtype):
    """Grids given as [43, n] / [39, n] arrays, as rows of a buffer at irregular offsets, and a batch
    mixing both all give the single-grid result bit for bit (the plan keeps one pointer per table
    entry whatever the layout)."""
    import paper_1804_10120_gb300 as tl
    td = torch.float32 if dtype == "f32" else torch.float64
    sides = [int(s) for s in np.random.default_rng(6).integers(3, 24, 30)]
    hosts, xs, ys = make_batch(sides, 24, td)
    refs = [tl.tl_dtg_forward(x, dtype=dtype) for x in xs]
    def scattered(count, n):
        # rows of one buffer at offsets that are not equally spaced
        offs = [k * (n + 64) + (k % 3) * 8 for k in range(count)]
        buf = torch.full((offs[-1] + n + 8,), float("nan"), dtype=td, device=dev())
        return [buf[o:o + n] for o in offs]
    rows_x = []
    for x in xs:
        r = scattered(43, x.shape[1])
        for k in range(43):
            r[k].copy_(x[k])
        rows_x.append(r)
    rows_y = [scattered(39, y.shape[1]) for y in ys]
    mixed_x = [rows_x[d] if d % 2 else xs[d] for d in range(len(xs))]
    mixed_y = [rows_y[d] if d % 2 else ys[d] for d in range(len(ys))]
    for bx, by in ((xs, ys), (rows_x, rows_y), (mixed_x, mixed_y)):
        for y in by:
            for r in (y if isinstance(y, list) else [y]):
                r.fill_(float("nan"))
        plan = tl.BatchPlan(bx, by, dtype=dtype)
        for ppt in (1, 4):
            plan.set_config(*plan.config, ppt)
            plan.launch()
            torch.cuda.synchronize()
            for y, r in zip(by, refs):
                got = torch.stack(y) if isinstance(y, list) else y
                assert torch.equal(got, r), (dtype, ppt)
        plan.check()
        plan.close()


STAGED = {"f64": [(128, 2), (128, 3), (256, 2)], "f32": [(128, 2), (128, 3), (256, 2), (256, 3), (512, 2)]}


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_staged_inputs_every_depth_bitwise(dtype):
    """Inputs staged through shared memory (depth 2 or 3) for every block size provided, at one and at
    the most blocks per SM: bit for bit the single-grid result on grids whose rows start on a 16-byte
    boundary (staged), whose rows do not (odd n in binary64 as [43, n] arrays: loaded directly), whose
    last tile has a byte length that is not a multiple of 16 (the rest of the tile loaded directly),
    a one-point and an empty grid; then in a CUDA graph."""
    import paper_1804_10120_gb300 as tl
    td = torch.float32 if dtype == "f32" else torch.float64
    sides = [8, 9, 1, 0, 13, 16, 7, 21, 4, 11, 6]
    hosts, xs, ys = make_batch(sides, 25, td)
    refs = [tl.tl_dtg_forward(x, dtype=dtype) for x in xs]
    torch.cuda.synchronize()
    plan = tl.BatchPlan(xs, ys, dtype=dtype)
    for threads, stages in STAGED[dtype]:
        plan.set_staging(0)                  # the block size is checked against the current depth
        plan.set_config(threads, 1, 1)
        plan.set_staging(stages)
        assert plan.staging == stages and plan.points_per_thread == 1
        for bps in (1, 99):
            if bps == 99:   # as many blocks per SM as the shared memory allows
                b = 1
                while True:
                    try:
                        plan.set_config(threads, b + 1)
                    except tl.TLError:
                        break
                    b += 1
                plan.set_config(threads, b)
            for y in ys:
                y.fill_(float("nan"))
            plan.launch()
            torch.cuda.synchronize()
            for d, (y, r) in enumerate(zip(ys, refs)):
                assert torch.equal(y, r), (dtype, threads, stages, bps, d)
    plan.check()
    assert tl.tl_wait_timeouts() == 0
    for y in ys:
        y.fill_(float("nan"))
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        plan.launch(stream=s)
    g.replay()
    torch.cuda.synchronize()
    for y, r in zip(ys, refs):
        assert torch.equal(y, r)
    plan.set_staging(0)
    assert plan.staging == 0
    plan.close()


def test_staging_rejects_what_is_not_provided():
    import paper_1804_10120_gb300 as tl
    hosts, xs, ys = make_batch([6, 5], 26)
    plan = tl.BatchPlan(xs, ys)
    plan.set_config(512, 1, 1)
    with pytest.raises(tl.TLError) as e:
        plan.set_staging(2)                  # 512 x 2 binary64 stages do not fit in shared memory
    assert e.value.status == 1
    plan.set_config(128, 1, 2)
    plan.set_staging(3)
    assert plan.points_per_thread == 1
    with pytest.raises(tl.TLError):
        plan.set_config(128, 1, 2)           # a staged plan computes one point per thread
    plan.close()
    plan = tl.BatchPlan(xs, ys, dtype="f64_ff")
    with pytest.raises(tl.TLError) as e:
        plan.set_staging(2)
    assert e.value.status == 3
    plan.close()


@pytest.mark.parametrize("dtype", ["f64", "f64_ff", "f32"])
def test_empty_and_one_point_grids_inside_a_batch(dtype):
    """Empty and one-point grids between ordinary ones, at every block size, blocks per SM and points
    per thread: each grid bit for bit the single-grid kernel's (the empty ones untouched), and the
    plan's status word clean."""
    import paper_1804_10120_gb300 as tl
    tdt = torch.float32 if dtype == "f32" else torch.float64
    sides = [0, 1, 0, 0, 5, 1, 0, 9, 0, 1, 3, 0]
    hosts, xs, ys = make_batch(sides, 31, dtype=tdt)
    refs = [tl.tl_dtg_forward(x, dtype=dtype) for x in xs]
    plan = tl.BatchPlan(xs, ys, dtype=dtype)
    torch.cuda.synchronize()
    ran = 0
    for threads in (128, 256, 512):
        for bps in (1, 2):
            for ppt in (1, 2, 4):
                try:
                    plan.set_config(threads, bps, ppt)
                except tl.TLError as e:          # beyond this kernel's occupancy
                    assert e.status == 1
                    continue
                for y in ys:
                    y.fill_(float("nan"))
                plan.launch()
                torch.cuda.synchronize()
                ran += 1
                for y, r in zip(ys, refs):
                    assert torch.equal(y.view(torch.int64 if dtype != "f32" else torch.int32),
                                       r.view(torch.int64 if dtype != "f32" else torch.int32)), (threads, bps, ppt)
    assert ran > 0
    plan.check()
    assert_components(ys[7].double().cpu().numpy(), oracle.forward(hosts[7]),
                      TOL_F64 if dtype != "f32" else 5e-6, what="9^3 grid")
    plan.close()
