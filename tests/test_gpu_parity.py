"""Stage-by-stage parity of the CUDA path (through the C ABI) against the
oracle on identical inputs: integer stages bit for bit, FP64 elevations within
1e-12 relative per step, FP32 elevations within the FP32 bound."""
import numpy as np
import pytest

import oracle
from paper_1803_02977_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL64 = 1e-12


def _lem():
    from paper_1803_02977_gb300 import lem
    return lem


def _dev():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return torch.device("cuda:0")


def _int_grid(nx, ny, seed, levels=5):
    u = synth.uniform01(seed, nx * ny).reshape(ny, nx)
    return np.floor(u * levels)


def _tilted(nx, ny, seed, slope=0.05):
    # a plane falling toward the west edge plus small noise: long flow paths,
    # many levels (exercises the narrow single-block mode and the wide mode)
    x = np.arange(nx, dtype=np.float64)[None, :]
    h = slope * 100.0 * x + 0.01 * synth.uniform01(seed, nx * ny).reshape(ny, nx)
    h[0, :] = h[-1, :] = h[:, 0] = h[:, -1] = 0.0
    return h


def _far_minima(nx, ny, seed):
    # neighbours far below a cell (zero, denormal, tiny) mixed with ones
    # just inside and just beyond 18 binades below it, singly and in pairs:
    # the receivers' high-word path takes one far group minimum as 0 and
    # must leave two far members, or any doubt, to the exact comparison
    h = 0.5 + synth.uniform01(seed, nx * ny).reshape(ny, nx)
    r = synth.uniform01(seed + 1, nx * ny).reshape(ny, nx)
    for lo, val in ((0.00, 0.0), (0.05, 5e-324), (0.08, 1e-300), (0.11, 2.0 ** -20),
                    (0.14, 2.0 ** -19), (0.17, 2.0 ** -19 * (1 - 2.0 ** -40)),
                    (0.20, 2.0 ** -18), (0.23, 2.0 ** -20 * (1 + 2.0 ** -21))):
        h[(r >= lo) & (r < lo + 0.03)] = val
    h[0, :] = h[-1, :] = h[:, 0] = h[:, -1] = 0.0
    return h


CASES = [
    ("3x3", lambda: synth.noise_surface(3, 3, 1)),
    ("5x4", lambda: synth.noise_surface(5, 4, 2)),
    ("17x13", lambda: synth.noise_surface(17, 13, 3)),
    ("64x64_int", lambda: _int_grid(64, 64, 4)),
    ("flat_40x30", lambda: np.zeros((30, 40))),
    ("plateau_50x50", lambda: np.pad(np.full((48, 48), 7.0), 1)),
    ("256x256", lambda: synth.noise_surface(256, 256, 1)),
    ("333x517", lambda: synth.noise_surface(333, 517, 5)),
    ("tilted_300x200", lambda: _tilted(300, 200, 6)),
    ("tilted_1500x64", lambda: _tilted(1500, 64, 7, slope=0.2)),
    ("1031x777_int", lambda: _int_grid(1031, 777, 8, levels=40)),
    ("far_minima_300x200", lambda: _far_minima(300, 200, 31)),
    # negative elevations (a surface below a datum): the codes pass redoes
    # every strip holding one with the exact per-cell form
    ("negative_157x212", lambda: np.random.default_rng(8).random((157, 212)) - 0.5),
    ("below_datum_300x200", lambda: _tilted(300, 200, 6) - 50.0),
    ("signed_zeros_90x70", lambda: _signed_zeros(90, 70, 12)),
]


def _run_stages(h_np, dtype=torch.float64, count_bits=32, **par):
    lem = _lem()
    dev = _dev()
    h = torch.tensor(h_np, dtype=dtype, device=dev).contiguous()
    mdl = lem.Model(h, count_bits=count_bits, **par)
    rec = mdl.receivers()
    dnum, donor = mdl.donors()
    q, lev, depth = mdl.levels()
    cnt = mdl.accumulate()
    mdl.erode()
    mdl.sync()
    out = dict(rec=rec.cpu().numpy(), dnum=dnum.cpu().numpy(), donor=donor.cpu().numpy(),
               queue=q.cpu().numpy(), levels=lev.cpu().numpy(), depth=depth.cpu().numpy(),
               cnt=cnt.cpu().numpy(), h=h.cpu().numpy())
    mdl.close()
    return out


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_stages_fp64_bit_exact_and_tolerance(name, make):
    h0 = make()
    par = dict(dx=100.0, K=1e-4, m=0.5, U=1e-3, dt=1000.0)
    g = _run_stages(h0, **par)
    ref = oracle.StepGraph(h0)
    assert np.array_equal(g["rec"], ref.rec)
    assert np.array_equal(g["dnum"], ref.dnum)
    assert np.array_equal(g["donor"], ref.donor)
    assert np.array_equal(g["queue"], ref.queue)
    assert np.array_equal(g["levels"], ref.levels)
    assert np.array_equal(g["depth"], ref.depth)
    assert np.array_equal(g["cnt"], ref.cnt)
    p = oracle.params(**par)
    want, _ = oracle.step(h0, p)
    scale = max(np.abs(want).max(), 1.0)
    assert np.abs(g["h"] - want).max() <= REL64 * scale


def _signed_zeros(nx, ny, seed):
    """Zeros of both signs among small positive values: -0.0 has the sign bit
    set, so a strip holding one takes the codes pass's checked form."""
    rng = np.random.default_rng(seed)
    h = rng.choice([0.0, -0.0, 0.25, 0.5, 1.0], (ny, nx))
    h[1::5, 2::7] = 3.0
    return h


def _adversarial(kind, nx, ny, seed):
    """Surfaces built to provoke FP64 rounding collisions between slopes."""
    rng = np.random.default_rng(seed)
    if kind == "tiny_next_to_large":
        h = rng.random((ny, nx)) * 2.0 ** -60
        h[1::3, 1::3] = 1.0 + rng.random(h[1::3, 1::3].shape)
    elif kind == "few_ulps":
        base = 1.0 + rng.random()
        h = base + rng.integers(0, 6, (ny, nx)) * np.spacing(base)
    elif kind == "mixed_zeros":
        h = rng.choice([0.0, 1e-300, 5e-324, 1e-17, 0.5, 1.0, 3.0], (ny, nx))
    elif kind == "low_bits":
        h = np.full((ny, nx), 1e-20) + rng.integers(0, 3, (ny, nx)) * 1e-36
        h[1::4, 1::4] = 1e3
    else:  # "negative_and_nan": the exact reference form handles these cells
        h = rng.random((ny, nx)) - 0.5
        h[rng.random((ny, nx)) < 0.01] = np.nan
        h[rng.random((ny, nx)) < 0.01] = -0.0
    return h


@pytest.mark.parametrize("kind", ["tiny_next_to_large", "few_ulps", "mixed_zeros", "low_bits",
                                  "negative_and_nan"])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_receivers_adversarial_rounding(kind, dtype):
    lem = _lem()
    dev = _dev()
    h0 = _adversarial(kind, 211, 157, 7)
    if dtype == "f32":
        h0 = h0.astype(np.float32)
    h = torch.tensor(h0, device=dev)
    mdl = lem.Model(h)
    rec = mdl.receivers().cpu().numpy()
    if kind == "negative_and_nan":
        # non-finite elevations are reported; the receivers are still written
        with pytest.raises(lem.LemError) as e:
            mdl.sync()
        assert e.value.status == lem.LEM_EINVAL
    else:
        mdl.sync()
    mdl.close()
    assert np.array_equal(rec, oracle.receivers(h0))


def _oracle_masks(rec, nx, ny):
    """Donor masks from a receiver array: bit k of cell c set iff its
    neighbour k drains into c (k = NW, N, NE, W, E, SW, S, SE)."""
    n = nx * ny
    d = np.arange(n)
    r = rec.astype(np.int64)
    sel = r != d
    dy = d[sel] // nx - r[sel] // nx
    dx = d[sel] % nx - r[sel] % nx
    # direction of the donor as seen from its receiver: (dy, dx) -> k
    table = np.array([0, 1, 2, 3, -1, 4, 5, 6, 7], np.int64)
    k = table[(dy + 1) * 3 + (dx + 1)]
    assert np.all(k >= 0)
    m = np.zeros(n, np.int64)
    np.bitwise_or.at(m, r[sel], 1 << k)
    return m.astype(np.uint8)


FP32_STEP_CASES = [
    ("3x3", lambda: synth.noise_surface(3, 3, 1)),
    ("5x4", lambda: synth.noise_surface(5, 4, 2)),
    ("61x67", lambda: synth.noise_surface(61, 67, 3)),
    # band edges: 130 = 2 bands of 60 + 10 columns, odd rows
    ("130x127", lambda: synth.noise_surface(130, 127, 4, south_tilt=1e-4)),
    ("512x300", lambda: synth.noise_surface(512, 300, 5)),
    # row pitch not a multiple of 16 bytes: chunks staged element-wise
    ("333x517_pitch", lambda: synth.noise_surface(333, 517, 6)),
    ("int_300x300", lambda: _int_grid(300, 300, 9, levels=12)),
    ("tilted_1500x64", lambda: _tilted(1500, 64, 7, slope=0.2)),
    ("far_minima_300x200", lambda: _far_minima(300, 200, 31)),
    ("tiny_next_to_large", lambda: _adversarial("tiny_next_to_large", 211, 157, 7)),
    ("few_ulps", lambda: _adversarial("few_ulps", 211, 157, 7)),
    ("mixed_zeros", lambda: _adversarial("mixed_zeros", 211, 157, 7)),
    ("low_bits", lambda: _adversarial("low_bits", 211, 157, 7)),
    ("negative", lambda: np.random.default_rng(8).random((157, 212)) - 0.5),
    ("below_datum_300x200", lambda: _tilted(300, 200, 6) - 50.0),
    ("signed_zeros_90x70", lambda: _signed_zeros(90, 70, 12)),
    ("grid2048_f32", lambda: synth.workload("grid2048_f32").initial()),
]


@pytest.mark.parametrize("name,make", FP32_STEP_CASES, ids=[c[0] for c in FP32_STEP_CASES])
def test_fp32_tiered_step_graph_and_elevations(name, make):
    """The tiered step's own Alg 1-2 pass on FP32 elevations (column bands,
    TMA chunk ring): the receivers and donor masks it used are the oracle's,
    bit for bit, and the new elevations are within the FP32 bound."""
    lem = _lem()
    dev = _dev()
    h32 = make().astype(np.float32)
    ny, nx = h32.shape
    par = dict(dx=100.0, K=2e-5, m=0.45, U=1e-3, dt=500.0)
    h = torch.tensor(h32, device=dev)
    mdl = lem.Model(h, **par)
    mdl.step(1)
    rec, msk = mdl.last_graph()
    mdl.sync()
    got_h = h.cpu().numpy().astype(np.float64)
    mdl.close()
    want_rec = oracle.receivers(h32)
    assert np.array_equal(rec.cpu().numpy(), want_rec)
    assert np.array_equal(msk.cpu().numpy(), _oracle_masks(want_rec, nx, ny))
    want, _ = oracle.step(h32.astype(np.float64), oracle.params(**par))
    tol = 4 * 2.0 ** -24 * np.maximum(np.abs(want), 1.0)
    assert np.all(np.abs(got_h - want) <= tol)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("value", [float("nan"), float("inf"), -float("inf")])
def test_nonfinite_elevation_stops_the_step(dtype, value):
    """A non-finite elevation is reported as LEM_EINVAL and the step changes
    no elevation; once the value is replaced, the context steps again."""
    lem = _lem()
    dev = _dev()
    h0 = synth.noise_surface(200, 150, 3)
    npt = np.float64 if dtype == "f64" else np.float32
    bad = h0.astype(npt)
    bad[70, 90] = value
    h = torch.tensor(bad, device=dev)
    mdl = lem.Model(h)
    mdl.step(1)
    with pytest.raises(lem.LemError) as e:
        mdl.sync()
    assert e.value.status == lem.LEM_EINVAL
    after = h.cpu().numpy()
    assert np.array_equal(np.isnan(after), np.isnan(bad))
    ok = ~np.isnan(bad)
    assert np.array_equal(after[ok], bad[ok])
    h.copy_(torch.tensor(h0.astype(npt), device=dev))
    mdl.step(1)
    mdl.sync()
    mdl.close()


def test_stages_int64_counts():
    h0 = synth.noise_surface(300, 211, 9)
    g = _run_stages(h0, count_bits=64)
    ref = oracle.StepGraph(h0)
    assert g["cnt"].dtype == np.int64
    assert np.array_equal(g["cnt"], ref.cnt)


@pytest.mark.parametrize("nx,ny,seed", [(256, 256, 1), (401, 173, 2), (64, 700, 3)])
def test_fp32_integer_stages_bit_exact_and_erosion_bound(nx, ny, seed):
    h32 = synth.noise_surface(nx, ny, seed).astype(np.float32)
    par = dict(dx=100.0, K=2e-5, m=0.45, U=1e-3, dt=500.0)
    g = _run_stages(h32, dtype=torch.float32, **par)
    ref = oracle.StepGraph(h32)  # receivers on the promoted FP32 values
    for key in ("rec", "dnum", "donor", "queue", "levels", "depth", "cnt"):
        assert np.array_equal(g[key], getattr(ref, key)), key
    want, _ = oracle.step(h32.astype(np.float64), oracle.params(**par))
    # FP32 increment form: a few units of FP32 rounding of the elevation
    tol = 4 * 2.0 ** -24 * np.maximum(np.abs(want), 1.0)
    assert np.all(np.abs(g["h"].astype(np.float64) - want) <= tol)


def test_step_matches_oracle_per_step():
    lem = _lem()
    dev = _dev()
    w = synth.workload("grid256_f64")
    p = oracle.params(dx=w.dx, K=w.K, m=w.m, U=w.U, dt=w.dt)
    h_np = w.initial()
    h = torch.tensor(h_np, device=dev)
    mdl = lem.Model(h, dx=w.dx, K=w.K, m=w.m, U=w.U, dt=w.dt)
    for _ in range(10):
        before = h.cpu().numpy()
        mdl.step(1)
        mdl.sync()
        want, _ = oracle.step(before, p)
        got = h.cpu().numpy()
        assert np.abs(got - want).max() <= REL64 * max(np.abs(want).max(), 1.0)
    # several steps in one launch equal the same steps launched one by one
    h2 = torch.tensor(h_np, device=dev)
    m2 = lem.Model(h2, dx=w.dx, K=w.K, m=w.m, U=w.U, dt=w.dt)
    m2.step(10)
    m2.sync()
    assert torch.equal(h, h2)
    mdl.close()
    m2.close()


# (name, grid, which lem_step tiers must run; None: not pinned)
STEP_CASES = [
    ("noise_256", lambda: synth.noise_surface(256, 256, 1), "tiles"),
    # row pitch not a multiple of 16 bytes: strips staged element-wise, not by TMA
    ("noise_odd_257x190", lambda: synth.noise_surface(257, 190, 4), "tiles"),
    ("noise_tilt_700x500", lambda: synth.noise_surface(700, 500, 3, south_tilt=1e-4), "tiles"),
    ("far_minima_300x200", lambda: _far_minima(300, 200, 31), None),
    ("int_300x300", lambda: _int_grid(300, 300, 9, levels=12), None),
    # one chain of ~300 cells per row, rooted on the west edge: too deep for a
    # warp's tile; the block or the device tier takes them, depending on how
    # many edge tiles one block claims
    ("tilted_300x64", lambda: _tilted(300, 64, 5, slope=0.2), None),
    # one basin of ~700 cells around a single pit: larger than a warp's queue,
    # within one block's, whichever block claims its tile
    ("funnel_256", lambda: _funnel(256, 256, 13), "block"),
    # chains of ~1500 cells (eight per edge tile): beyond the block's share too
    ("tilted_1500x64", lambda: _tilted(1500, 64, 7, slope=0.2), "device"),
    # a cone draining the whole grid to one outlet: one tree of ~90k cells
    ("cone_300x300", lambda: _cone(300, 300, 11), "device"),
]


def _funnel(nx, ny, seed, cx=48, cy=44, r=15.0):
    h = 100.0 + synth.uniform01(seed, nx * ny).reshape(ny, nx)
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    d = np.hypot(x - cx, y - cy)
    inside = d <= r
    h[inside] = 50.0 + d[inside] + 0.001 * h[inside]
    h[0, :] = h[-1, :] = h[:, 0] = h[:, -1] = 0.0
    return h


def _cone(nx, ny, seed):
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    cy = ny // 2
    h = 100.0 * np.hypot(x, y - cy) + 0.01 * synth.uniform01(seed, nx * ny).reshape(ny, nx)
    h[0, :] = h[-1, :] = h[:, 0] = h[:, -1] = 1e6  # raised rim ...
    h[cy, 0] = 0.0                                 # ... but for one outlet
    return h


@pytest.mark.parametrize("name,make,path", STEP_CASES, ids=[c[0] for c in STEP_CASES])
def test_step_modes_match_oracle_and_each_other(name, make, path):
    lem = _lem()
    dev = _dev()
    h0 = make()
    par = dict(dx=100.0, K=2e-5, m=0.5, U=1e-3, dt=1000.0)
    p = oracle.params(**par)
    hs = {}
    jumped = 0
    for mode in (0, 1):
        h = torch.tensor(h0, device=dev)
        mdl = lem.Model(h, **par)
        lem.lem_set_step_mode(mdl.ctx, mode)
        cur = h0.copy()
        for _ in range(4):
            mdl.step(1)
            mdl.sync()
            want, _ = oracle.step(cur, p)
            got = h.cpu().numpy()
            assert np.abs(got - want).max() <= REL64 * max(np.abs(want).max(), 1.0)
            cur = got
        priv, wide = lem.lem_step_stats(mdl.ctx)
        tiers = lem.lem_tier_stats(mdl.ctx)
        if mode == 1:
            # device-wide mode does not use the tiered form
            assert (priv, wide) == (0, 0) and tiers == (0, 0, 0)
        else:
            assert sum(tiers) == 4 * h0.size  # every cell handled once per step
            if path == "tiles":
                assert tiers[1] == tiers[2] == 0 and (priv, wide) == (4, 0)
            elif path == "block":
                assert tiers[1] > 0 and tiers[2] == 0 and (priv, wide) == (4, 0)
            elif path == "device":
                assert tiers[2] > 0 and wide >= 1
            jumped = lem.lem_jump_stats(mdl.ctx)[0]
        hs[mode] = h.cpu().numpy()
        mdl.close()
    if jumped == 0:
        # same per-cell arithmetic in both forms: identical elevations
        assert np.array_equal(hs[0], hs[1])
    else:
        # deep trees were eroded by composing the updates along the receivers
        # (another association order of the same sums): within the tolerance
        assert np.abs(hs[0] - hs[1]).max() <= REL64 * max(np.abs(hs[1]).max(), 1.0)


def test_uplift_field():
    lem = _lem()
    dev = _dev()
    nx, ny = 120, 90
    h0 = synth.noise_surface(nx, ny, 21)
    Uf = 1e-3 * (1.0 + 0.5 * synth.signed_field(nx, ny, 22))
    par = dict(dx=100.0, K=3e-5, m=0.5, U=0.0, dt=1000.0)
    h = torch.tensor(h0, device=dev)
    mdl = lem.Model(h, **par)
    mdl.set_uplift_field(torch.tensor(Uf, device=dev))
    mdl.step(1)
    mdl.sync()
    want, _ = oracle.step(h0, oracle.params(**dict(par, Ufield=Uf)))
    assert np.abs(h.cpu().numpy() - want).max() <= REL64 * np.abs(want).max()


def test_frozen_channel_closed_form():
    lem = _lem()
    dev = _dev()
    nx = 200
    dx, K, m, U, dt = 100.0, 1e-5, 0.5, 1e-3, 1000.0
    rec = np.arange(3 * nx, dtype=np.int32)
    for x in range(1, nx - 1):
        rec[nx + x] = nx + x - 1
    area = dx * dx
    prof = np.zeros((3, nx))
    for x in range(1, nx - 1):
        prof[1, x] = prof[1, x - 1] + dx * U / (K * ((nx - 1 - x) * area) ** m)
    h = torch.tensor(prof, device=dev)
    mdl = lem.Model(h, dx=dx, K=K, m=m, U=U, dt=dt)
    mdl.set_receivers(torch.tensor(rec, device=dev))
    mdl.step(3)
    mdl.sync()
    assert np.abs(h.cpu().numpy() - prof).max() <= 1e-12 * prof.max()
    q, lev, depth = mdl.levels()
    assert lev.numel() == nx  # level 0 plus one level per chain cell: L = nx-1
    mdl.close()


def test_frozen_cycle_is_reported():
    lem = _lem()
    dev = _dev()
    nx, ny = 6, 5
    rec = np.arange(nx * ny, dtype=np.int32)
    a, b = 2 * nx + 2, 2 * nx + 3
    rec[a], rec[b] = b, a  # two interior cells draining into each other
    h = torch.zeros((ny, nx), dtype=torch.float64, device=dev)
    mdl = lem.Model(h)
    mdl.set_receivers(torch.tensor(rec, device=dev))
    with pytest.raises(lem.LemError) as e:
        mdl.levels()
    assert e.value.status == lem.LEM_EINVAL
    # the tiered step reaches no cell of the cycle either
    with pytest.raises(lem.LemError) as e:
        mdl.step(1)
        mdl.sync()
    assert e.value.status == lem.LEM_EINVAL
    bad = np.arange(nx * ny, dtype=np.int32)
    bad[2 * nx + 2] = 0  # not a neighbour
    with pytest.raises(lem.LemError) as e:
        mdl.set_receivers(torch.tensor(bad, device=dev))
    assert e.value.status == lem.LEM_EINVAL
    mdl.close()


def test_state_errors_and_timeout_path():
    lem = _lem()
    dev = _dev()
    h = torch.tensor(synth.noise_surface(32, 32, 3), device=dev)
    mdl = lem.Model(h)
    with pytest.raises(lem.LemError) as e:
        mdl.levels()
    assert e.value.status == lem.LEM_ESTATE
    with pytest.raises(lem.LemError) as e:
        mdl.erode()
    assert e.value.status == lem.LEM_ESTATE
    lem.lem_set_wait_limit(mdl.ctx, 0.02)
    assert lem.lem_selftest_wait(mdl.ctx) == lem.LEM_ETIMEOUT
    lem.lem_set_wait_limit(mdl.ctx, 2.0)
    # the context stays usable after the timed-out wait
    before = h.cpu().numpy()
    mdl.step(1)
    mdl.sync()
    want, _ = oracle.step(before, oracle.params())
    assert np.abs(h.cpu().numpy() - want).max() <= REL64 * np.abs(want).max()
    mdl.close()


def test_determinism_repeat():
    lem = _lem()
    dev = _dev()
    h_np = synth.noise_surface(700, 500, 44)
    outs = []
    for _ in range(2):
        h = torch.tensor(h_np, device=dev)
        mdl = lem.Model(h)
        mdl.receivers()
        q, lev, _ = mdl.levels(want_depth=False)
        cnt = mdl.accumulate()
        mdl.erode()
        mdl.sync()
        outs.append((q.cpu(), lev.cpu(), cnt.cpu(), h.cpu()))
        mdl.close()
    for a, b in zip(outs[0], outs[1]):
        assert torch.equal(a, b)
