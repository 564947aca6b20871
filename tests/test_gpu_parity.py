"""GPU parity: the CUDA library (through its C ABI) against the CPU oracle,
element by element on the same seeded inputs.

Sizes span several 8^3 bricks and ragged tails; the oracle finishes each case
in seconds.  Tolerances: max |dT| <= 1e-12 max|T| (fp64), 2e-5 max|T| (fp32),
with identical tags (identical accepted sets)."""
import math
import time

import numpy as np
import pytest
import torch

from paper_1502_07303_gb300 import workloads as wl
from parity_util import compare

pytestmark = pytest.mark.gpu

DT = {"f32": torch.float32, "f64": torch.float64}


@pytest.fixture(scope="module")
def fmm():
    if not torch.cuda.is_available():
        pytest.fail("CUDA is required for the gpu tests")
    from paper_1502_07303_gb300 import fmm as _fmm
    return _fmm


def _dev(a, dt):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda", dtype=DT[dt])


def _host(t):
    return t.detach().cpu().numpy()


def _quantise(a, dt):
    """The input the GPU sees, as fp64 for the oracle."""
    return np.asarray(a, dtype=np.float32).astype(np.float64) if dt == "f32" else np.asarray(a, np.float64)


def run_sources(fmm, oracle, shape, h, src, speed, dt, **kw):
    sp_gpu = None if speed is None or np.isscalar(speed) else _dev(speed, dt)
    sp_const = speed if np.isscalar(speed) else None
    with fmm.Solver(shape, h, dtype=DT[dt], speed=sp_gpu if sp_gpu is not None else sp_const,
                    sources=src, **kw) as s:
        T, G = s.solve()
        stats = s.stats()
    sp_ref = None if speed is None else (speed if np.isscalar(speed) else _quantise(speed, dt))
    width = kw.get("width", math.inf)
    ref = oracle.solve_sources(shape, src, h, speed=sp_ref, width=width)
    return _host(T), _host(G), ref, stats


def run_reinit(fmm, oracle, phi, h, dt, **kw):
    phi_q = _quantise(phi, dt)
    with fmm.Solver(phi.shape, h, dtype=DT[dt], **kw) as s:
        T, G = s.reinit(_dev(phi, dt))
        stats = s.stats()
    ref = oracle.solve_reinit(phi_q, h, width=kw.get("width", math.inf))
    return _host(T), _host(G), ref, stats


# ---------------------------------------------------------------------------
# point sources, constant speed
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_point_source_64(fmm, oracle, dt):
    p = wl.point_source(64)
    T, G, ref, st = run_sources(fmm, oracle, p.shape, p.h, p.sources, None, dt)
    compare(T, G, ref, dt)
    assert st["error_flags"] == 0


@pytest.mark.parametrize("shape", [(16, 16, 16), (33, 17, 9), (7, 13, 40), (1, 1, 1), (1, 5, 1),
                                   (9, 9, 9)])
@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_sources_shapes(fmm, oracle, shape, dt):
    rng = np.random.default_rng(sum(shape))
    src = wl.random_cells(rng, shape, min(3, int(np.prod(shape))))
    h = wl.spacing(shape)
    T, G, ref, _ = run_sources(fmm, oracle, shape, h, src, 1.7, dt)
    compare(T, G, ref, dt)


@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_no_sources_all_far(fmm, oracle, dt):
    shape = (10, 12, 9)
    T, G, ref, st = run_sources(fmm, oracle, shape, 0.1, np.zeros((0, 3), np.int64), None, dt)
    assert np.all(G == 0) and np.all(np.isinf(T))
    compare(T, G, ref, dt)


# ---------------------------------------------------------------------------
# heterogeneous speed
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n", [24, 41])
@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_fourier_speed(fmm, oracle, n, dt):
    p = wl.fourier_sources(n=n, n_sources=4, n_receivers=8, seed=3)
    T, G, ref, st = run_sources(fmm, oracle, p.shape, p.h, p.sources, p.speed, dt)
    compare(T, G, ref, dt)


@pytest.mark.parametrize("schedule", [1, 2, 3])
def test_fourier_speed_many_seeds(fmm, oracle, schedule):
    """Twelve seeds, each solved twice: brick marches run concurrently, so the
    order in which halo values and their change flags reach a brick differs
    from run to run; every run must reach the oracle's fixed point."""
    for seed in range(12):
        p = wl.fourier_sources(n=41, n_sources=4, n_receivers=8, seed=seed)
        ref = oracle.solve_sources(p.shape, p.sources, p.h, speed=p.speed)
        sp = _dev(p.speed, "f64")
        for _ in range(2):
            with fmm.Solver(p.shape, p.h, dtype=torch.float64, speed=sp, sources=p.sources,
                            schedule=schedule) as s:
                T, G = s.solve()
            compare(_host(T), _host(G), ref, "f64")


@pytest.mark.parametrize("case", [4, 5])
def test_paper_speed_cases(fmm, oracle, case):
    """Sec. 5.1 cases 4 and 5 (Eq. (9), (10)): point source at the centre."""
    n = 40
    shape = (n, n, n)
    F = wl.paper_speed(shape, case)
    T, G, ref, _ = run_sources(fmm, oracle, shape, 1.0 / n, [(n // 2, n // 2, n // 2)], F, "f64")
    compare(T, G, ref, "f64")


# ---------------------------------------------------------------------------
# two-sided reinitialisation
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("shape", [(32, 32, 32), (29, 41, 23)])
@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_reinit_spheres(fmm, oracle, shape, dt):
    p = wl.random_spheres(shape=shape, count=6, seed=7)
    T, G, ref, _ = run_reinit(fmm, oracle, p.phi0, p.h, dt)
    compare(T, G, ref, dt)


def test_reinit_single_sphere_64(fmm, oracle):
    p = wl.single_sphere(64)
    T, G, ref, _ = run_reinit(fmm, oracle, p.phi0, p.h, "f64")
    compare(T, G, ref, "f64")


# ---------------------------------------------------------------------------
# restart parameters, narrow band, restart counts
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("stride", [0.5, 1.0, 2.0, 3.5, math.inf])
@pytest.mark.parametrize("bucket", [1.0, math.inf])
@pytest.mark.parametrize("schedule", [1, 2, 3])
def test_stride_bucket_schedule_do_not_change_the_result(fmm, oracle, stride, bucket, schedule):
    p = wl.random_spheres(shape=(40, 40, 40), count=5, seed=11)
    T, G, ref, _ = run_reinit(fmm, oracle, p.phi0, p.h, "f64", stride=stride, bucket=bucket,
                              schedule=schedule)
    compare(T, G, ref, "f64")


@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_phased_schedule_heterogeneous(fmm, oracle, dt):
    p = wl.fourier_sources(n=33, n_sources=4, n_receivers=8, seed=5)
    T, G, ref, st = run_sources(fmm, oracle, p.shape, p.h, p.sources, p.speed, dt, schedule=1,
                                exchange_passes=1)
    compare(T, G, ref, dt)


@pytest.mark.parametrize("dt", ["f64", "f32"])
@pytest.mark.parametrize("schedule", [0, 1, 3])
def test_narrow_band_width(fmm, oracle, dt, schedule):
    p = wl.random_spheres(shape=(36, 36, 36), count=4, seed=5)
    width = 0.08
    T, G, ref, _ = run_reinit(fmm, oracle, p.phi0, p.h, dt, width=width, schedule=schedule)
    compare(T, G, ref, dt, width=width)


@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_continuous_schedule_shapes(fmm, oracle, dt):
    for shape in [(16, 16, 16), (33, 17, 9), (1, 5, 1), (9, 9, 9)]:
        rng = np.random.default_rng(sum(shape))
        src = wl.random_cells(rng, shape, min(3, int(np.prod(shape))))
        T, G, ref, _ = run_sources(fmm, oracle, shape, wl.spacing(shape), src, 1.7, dt,
                                   schedule=3, stride=2.0)
        compare(T, G, ref, dt)


@pytest.mark.parametrize("schedule", [1, 2])
def test_single_brick_infinite_stride_two_restarts(fmm, oracle, schedule):
    """Sec. 5.3: with stride = inf one subdomain finishes in two restarts (the
    second only finds nothing left to do)."""
    shape = (8, 8, 8)
    T, G, ref, st = run_sources(fmm, oracle, shape, 1.0 / 8, [(1, 2, 3)], None, "f64",
                                stride=math.inf, schedule=schedule)
    compare(T, G, ref, "f64")
    assert st["restarts"] == 2


def test_restarts_scale_inversely_with_stride(fmm, oracle):
    """Sec. 5.4: nr is about proportional to nh / delta_s."""
    p = wl.point_source(48)
    nr = {}
    for stride in (1.0, 4.0):
        with fmm.Solver(p.shape, p.h, dtype=torch.float64, sources=p.sources, stride=stride,
                        schedule=1) as s:
            s.solve()
            nr[stride] = s.stats()["restarts"]
    assert nr[1.0] > 2.5 * nr[4.0]


def test_repeat_solve_same_handle(fmm, oracle):
    p = wl.point_source(24)
    with fmm.Solver(p.shape, p.h, dtype=torch.float64, sources=p.sources) as s:
        T1, G1 = s.solve()
        T2, G2 = s.solve()
    assert torch.equal(G1, G2)
    ref = oracle.solve_sources(p.shape, p.sources, p.h)
    compare(_host(T2), _host(G2), ref, "f64")


def test_invalid_speed_rejected(fmm):
    shape = (8, 8, 8)
    F = torch.ones(shape, dtype=torch.float64, device="cuda")
    F[3, 3, 3] = -1.0
    with pytest.raises(fmm.FmmError) as e:
        fmm.Solver(shape, 0.1, dtype=torch.float64, speed=F, sources=[(0, 0, 0)])
    assert e.value.code == fmm.FMM_ERR_INVALID
    F[3, 3, 3] = float("nan")
    with pytest.raises(fmm.FmmError):
        fmm.Solver(shape, 0.1, dtype=torch.float64, speed=F, sources=[(0, 0, 0)])


def test_restart_limit_reports_timeout(fmm):
    p = wl.point_source(32)
    with fmm.Solver(p.shape, p.h, dtype=torch.float64, sources=p.sources, stride=0.5,
                    max_restarts=3) as s:
        with pytest.raises(fmm.FmmError) as e:
            s.solve()
        assert e.value.code == fmm.FMM_ERR_TIMEOUT


@pytest.mark.parametrize("schedule", [1, 2, 3])
def test_kernel_timing_and_trace(fmm, oracle, schedule):
    """time_kernels: march time, one trace entry per march launch that did
    work, and the same result as without timing."""
    p = wl.random_spheres(shape=(48, 40, 44), count=5, seed=8)
    phi = _dev(p.phi0, "f64")
    for rep in range(2):                      # the event pool is reused
        with fmm.Solver(p.shape, p.h, dtype=torch.float64, schedule=schedule, stride=4.0,
                        time_kernels=True) as s:
            T, G = s.reinit(phi)
            st = s.stats()
            tr = s.trace()
        assert st["march_ms"] > 0.0 and st["march_launches"] >= 1
        assert len(tr) == st["march_launches"]
        assert all(ms >= 0.0 for _, _, _, ms in tr) and sum(b for _, _, b, _ in tr) > 0
        assert st["restarts"] >= 2 and st["error_flags"] == 0
    compare(_host(T), _host(G), oracle.solve_reinit(p.phi0, p.h), "f64")


@pytest.mark.parametrize("schedule", [2, 3])
def test_device_wait_limit_reports_timeout_and_recovers(fmm, oracle, schedule):
    """A device wait that runs out (the brick queue held open by one phantom
    pending brick) sets an error bit, the call returns FMM_ERR_TIMEOUT after
    about wait_limit_ms, and the GPU and the library stay usable."""
    p = wl.random_spheres(shape=(32, 32, 32), count=3, seed=4)
    phi = _dev(p.phi0, "f64")
    t0 = time.perf_counter()
    with fmm.Solver(p.shape, p.h, dtype=torch.float64, schedule=schedule, wait_limit_ms=50,
                    hold_queue=1) as s:
        with pytest.raises(fmm.FmmError) as e:
            s.reinit(phi)
        assert e.value.code == fmm.FMM_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 60
    T, G, ref, _ = run_reinit(fmm, oracle, p.phi0, p.h, "f64", schedule=schedule)
    compare(T, G, ref, "f64")


@pytest.mark.parametrize("dt", ["f64", "f32"])
@pytest.mark.parametrize("schedule", [1, 2, 3])
def test_paper_case6_obstacles(fmm, oracle, dt, schedule):
    """Sec. 5.1 case 6: point source at the centre, four concentric spherical
    shells of F = 0 with gaps (Eq. (11)); obstacle cells stay FAR."""
    n = 48
    shape = (n, n, n)
    F = wl.paper_speed(shape, 6)
    T, G, ref, _ = run_sources(fmm, oracle, shape, 1.0 / n, [(n // 2, n // 2, n // 2)], F, dt,
                               schedule=schedule)
    compare(T, G, ref, dt)
    assert np.all(G[F == 0.0] == 0) and np.all(np.isinf(T[F == 0.0]))
    assert np.all(G[F > 0.0] >= 2)   # every open cell is reached through the gaps


@pytest.mark.parametrize("dt", ["f64", "f32"])
@pytest.mark.parametrize("schedule", [1, 2, 3])
def test_paper_case2_plane(fmm, oracle, dt, schedule):
    """Sec. 5.1 case 2: the plane 100x + y + 2z = 0 through the centre of the
    [-0.5, 0.5]^3 cube, positive where 100x + y + 2z > 0; every cell depends
    on three upwind cells of the same pattern, so information crosses each
    x plane corner to corner in strict order."""
    n = 40
    shape = (n, n, n)
    h = 1.0 / n
    c = (np.arange(n) + 0.5) * h - 0.5
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    phi = (100 * x + y + 2 * z) / math.sqrt(100 ** 2 + 1 + 4)
    T, G, ref, _ = run_reinit(fmm, oracle, phi, h, dt, schedule=schedule)
    compare(T, G, ref, dt)


@pytest.mark.parametrize("dt", ["f64", "f32"])
@pytest.mark.parametrize("schedule", [1, 2, 3])
@pytest.mark.parametrize("hetero", [False, True])
def test_tape_and_tape_free_kernels_agree(fmm, oracle, dt, schedule, hetero):
    """The march kernels are compiled twice, with and without recording the
    upwind sets for the adjoint; the set codes never feed back into psi, so
    both forward solves reach the oracle's fixed point on every schedule
    (point sources, constant and heterogeneous speed; two-sided
    reinitialisation)."""
    p = wl.fourier_sources(n=37, n_sources=4, n_receivers=8, seed=11)
    speed = p.speed if hetero else 1.0
    for tape in (False, True):
        T, G, ref, st = run_sources(fmm, oracle, p.shape, p.h, p.sources, speed, dt,
                                    schedule=schedule, record_tape=tape)
        compare(T, G, ref, dt)
        assert st["error_flags"] == 0
    q = wl.random_spheres(n=29, count=5, seed=4)
    for tape in (False, True):
        T, G, ref, _ = run_reinit(fmm, oracle, q.phi0, q.h, dt, schedule=schedule,
                                  record_tape=tape)
        compare(T, G, ref, dt)


@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_reinit_degenerate_level_sets(fmm, oracle, dt):
    """Level sets without a front (one sign everywhere: every cell stays FAR,
    psi = +inf on either side as Algorithm 8 initialises it) and with exact
    zeros (a zero cell is an interface cell with psi = 0, sign +,
    Algorithm 8), against the oracle."""
    shape = (11, 9, 14)
    h = wl.spacing(shape)
    for phi in (np.full(shape, 0.3), np.full(shape, -0.2)):
        T, G, ref, _ = run_reinit(fmm, oracle, phi, h, dt)
        assert np.all(G == 0)
        assert np.all(T == np.inf)
        compare(T, G, ref, dt)
    x = (np.arange(shape[2]) + 0.5) * h
    phi = np.broadcast_to(np.round((x - 7.5 * h) / h)[None, None, :] * h, shape).copy()  # zeros at i = 7
    T, G, ref, _ = run_reinit(fmm, oracle, phi, h, dt)
    assert np.all(T[:, :, 7] == 0) and np.all(G[:, :, 7] == 3)
    compare(T, G, ref, dt)
