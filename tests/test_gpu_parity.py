"""GPU-vs-oracle parity of the CUDA path, called through the C ABI.

FP64 bar (relative L2 per variable, ||gpu - oracle|| / ||oracle||): 1e-12 on states
after the stated steps and on tendencies of non-steady states.  Both sides take the
same input state (the oracle's cell averages, copied to the device).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from synth import noise_field, perturb_h  # noqa: E402


def rh_perturbed(o, seed=0):
    """Rossby-Haurwitz state with seeded 1% cell-wise h noise: large, well-conditioned
    tendencies everywhere (the noise makes the flux divergence O(noise) relative)."""
    return np.ascontiguousarray(perturb_h(o.rossby_haurwitz(), noise_field((6, o.N, o.N), seed)))


@pytest.fixture(scope="module")
def hp():
    import paper_2411_19185_gb300 as hp
    hp.load()
    return hp


def rel_l2(a, b):
    return [float(np.linalg.norm(a[v] - b[v]) / np.linalg.norm(b[v])) for v in range(3)]


def to_dev(q, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(q)).to("cuda", dtype)


@pytest.mark.parametrize("case", ["geo", "rh", "dam", "bumps"])
def test_initial_conditions_match(hp, case):
    """Cell averages of the analytic cases (section 5): device kernel vs oracle."""
    N, k = 20, 5
    s = hp.Sphere(N, k)
    o = O.Oracle(N, k)
    cent = [(0.3, 0.2), (2.0, -0.7), (-1.5, 1.1)]
    if case == "geo":
        a, b = s.geostrophic(np.pi / 4), o.geostrophic(np.pi / 4)
    elif case == "rh":
        a, b = s.rossby_haurwitz(), o.rossby_haurwitz()
    elif case == "dam":
        a, b = s.dam_break(), o.dam_break()
    else:
        a, b = s.bumps(cent), o.bumps(cent)
    torch.cuda.synchronize()
    a = a.cpu().numpy()
    scale = [np.linalg.norm(b[v]) + 1e-300 for v in range(3)]
    err = [np.linalg.norm(a[v] - b[v]) / scale[v] if scale[v] > 1e-200 else np.abs(a[v]).max() for v in range(3)]
    assert max(err) < 1e-13, err


@pytest.mark.parametrize("k,N,tilt", [(3, 13, 0.0), (5, 20, 0.0), (7, 17, 0.3), (9, 24, 0.0), (11, 23, 0.0)])
def test_tendency_tpp_fp64(hp, k, N, tilt):
    """One evaluation of L(q) (eq. 3.1), TPP, FP64, several tiles with ragged tails."""
    s = hp.Sphere(N, k, coriolis_tilt=tilt)
    o = O.Oracle(N, k, coriolis_tilt=tilt)
    q = rh_perturbed(o)
    d = s.tendency(to_dev(q)).cpu().numpy()
    ref = o.tendency(q)
    assert max(rel_l2(d, ref)) < 1e-12, rel_l2(d, ref)
    assert s.status() == 0


def test_config1_c32_tpp5_10_steps(hp):
    """C32, TPP5, steady geostrophic flow (alpha = 0), SSP-RK3 dt = 600 s, 10 steps."""
    N, k = 32, 5
    s = hp.Sphere(N, k)
    o = O.Oracle(N, k)
    q0 = o.geostrophic(0.0)
    q = to_dev(q0)
    m0 = s.mass(q)
    s.step(q, 600.0, 10)
    ref = o.step(q0, 600.0, 10)
    got = q.cpu().numpy()
    assert max(rel_l2(got, ref)) < 1e-12, rel_l2(got, ref)
    m1 = s.mass(q)
    assert abs(m1 - m0) / abs(m0) < 1e-14
    assert abs(m1 - o.mass(ref)) / abs(m0) < 1e-14
    assert s.status() == 0


def test_wsrk3_steps(hp):
    """Wicker-Skamarock RK3 (eqs. 3.39-3.41) on a Rossby-Haurwitz state."""
    N, k = 16, 7
    s = hp.Sphere(N, k, rk=hp.HOPE_WSRK3)
    o = O.Oracle(N, k)
    q0 = o.rossby_haurwitz()
    q = to_dev(q0)
    s.step(q, 900.0, 3)
    ref = o.step(q0, 900.0, 3, O.WSRK3)
    assert max(rel_l2(q.cpu().numpy(), ref)) < 1e-12


def test_config2_c90_tpp11_full_size_one_step(hp):
    """Full-size C90 TPP11 (alpha = pi/4), the benchmark's launch configuration
    (graph-replayed SSP-RK3 step, dt = 300 s): one step against the oracle."""
    N, k = 90, 11
    s = hp.Sphere(N, k, coriolis_tilt=np.pi / 4)
    o = O.Oracle(N, k, coriolis_tilt=np.pi / 4)
    q0 = o.geostrophic(np.pi / 4)
    q = to_dev(q0)
    s.step(q, 300.0, 1)
    ref = o.step(q0, 300.0, 1)
    assert max(rel_l2(q.cpu().numpy(), ref)) < 1e-12
    assert s.status() == 0


def test_ghost_operator_size(hp):
    s = hp.Sphere(32, 5)
    nnz, rows = s.ghost_nnz()
    assert rows == 6 * (36 * 36 - 32 * 32)
    assert rows * 9 <= nnz < rows * 2000


def test_nonphysical_state_sets_status(hp):
    """phi <= 0 reaching the flux's sqrt (eq. 3.35) is reported through the sticky
    status word, not hidden."""
    N, k = 12, 3
    s = hp.Sphere(N, k)
    o = O.Oracle(N, k)
    q = o.rossby_haurwitz()
    q[0, 2, 5, 5] = -abs(q[0, 2, 5, 5])
    s.tendency(to_dev(q))
    st = s.status()
    assert st & hp._lib.HOPE_STATUS_NONPHYS_PHI
    assert s.status() == 0  # cleared by the read


def test_host_buffers_end_to_end(hp):
    """hope_step_host: host in, host out, copies inside the call."""
    N, k = 12, 5
    s = hp.Sphere(N, k)
    o = O.Oracle(N, k)
    q0 = o.rossby_haurwitz()
    qh = torch.from_numpy(q0.copy()).pin_memory()
    out = s.step_host(qh, 600.0, 2)
    ref = o.step(q0, 600.0, 2)
    assert max(rel_l2(out.numpy(), ref)) < 1e-12
