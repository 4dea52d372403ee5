"""GPU-vs-oracle parity of the bottom-topography path (eqs. 2.13-2.14, section 5.2's
mountain), called through the C ABI.

FP64 bar: relative L2 per variable 1e-11 on tendencies and 1e-12 on states.  The other
FP64 parity tests hold tendencies to 1e-12; here psi_B's per-cell weights are assembled
on the host as sums of k^2 products whose terms exceed the sum by up to ~1e3 (the
derivative weights of a k-point stencil alternate in sign), so the assembly's rounding
reaches ~1e-13 relative and 1e-11 keeps a factor 100.  FP32: 1e-4 on tendencies, the
flat FP32 path's bound.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from synth import noise_field, perturb_h  # noqa: E402

G = O.GRAVITY
H0, U0 = 5960.0, 20.0  # section 5.2


@pytest.fixture(scope="module")
def hp():
    import paper_2411_19185_gb300 as hp
    hp.load()
    return hp


def rel_l2(a, b):
    return [float(np.linalg.norm(a[v] - b[v]) / np.linalg.norm(b[v])) for v in range(3)]


def to_dev(q, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(q)).to("cuda", dtype)


def mountain_case(N, k, noise_seed=None, scheme=O.TPP):
    """Oracle with the mountain of eq. 5.8, the flow of section 5.2 (optionally with seeded
    1% depth noise for large tendencies everywhere) and the surface's cell averages."""
    o = O.Oracle(N, k, scheme=scheme)
    o.set_mountain()
    q = o.geostrophic(u0=U0, phi0=H0 * G)
    if noise_seed is not None:
        q = np.ascontiguousarray(perturb_h(q, noise_field((6, N, N), noise_seed)))
    return o, q, o.topography()


def test_mountain_initial_conditions_match(hp):
    """Device cell averages of section 5.2's surface (eq. 5.8) and of the flow over it
    (phi of eq. 5.1 read as the free surface) against the oracle's."""
    N, k = 20, 5
    s = hp.Sphere(N, k)
    o = O.Oracle(N, k)
    o.set_mountain()
    surf = s.mountain_surface().cpu().numpy()
    flow = s.mountain_flow().cpu().numpy()
    ref_s, ref_q = o.topography(), o.geostrophic(u0=U0, phi0=H0 * G)
    assert np.max(np.abs(surf - ref_s)) < 1e-13 * np.max(np.abs(ref_s))
    assert np.linalg.norm(flow[0] - ref_q[0]) < 1e-13 * np.linalg.norm(ref_q[0])
    assert np.linalg.norm(flow[1:] - ref_q[1:]) < 1e-13 * np.linalg.norm(ref_q[1:])


@pytest.mark.parametrize("k,N,scheme", [(3, 13, "tpp"), (5, 20, "tpp"), (7, 17, "tpp"), (11, 23, "tpp"),
                                        (3, 13, "weno"), (5, 20, "weno"), (7, 17, "weno"), (9, 18, "weno")])
def test_tendency_over_mountain_fp64(hp, k, N, scheme):
    """L(q) with the surface (eq. 3.1 with eqs. 2.13-2.14), FP64, ragged tiles; TPP, and the
    genuine-2D WENO-Z reconstructing sqrtG phi_t = depth + surface and subtracting the
    surface's own TPP values at the points (reading c26; the WENO FP64 contexts' balanced
    tile shapes)."""
    o, q, sbar = mountain_case(N, k, noise_seed=3, scheme=O.TPP if scheme == "tpp" else O.WENO)
    s = hp.Sphere(N, k, scheme=hp.HOPE_TPP if scheme == "tpp" else hp.HOPE_WENO2D)
    s.set_topography(sbar)
    d = s.tendency(to_dev(q)).cpu().numpy()
    ref = o.tendency(q)
    assert max(rel_l2(d, ref)) < 1e-11, rel_l2(d, ref)
    assert s.status() == 0
    # TPP adds psi_B in the reconstruction's epilogue; WENO2D runs a separate source kernel
    assert s.launches_per_stage() == (4 if scheme == "tpp" else 5)


def test_steps_over_mountain_fp64(hp):
    """SSP-RK3 steps of section 5.2's flow (C16, TPP5, dt = 600 s): a step graph captured
    before the surface is set is not replayed after it; states against the oracle and the
    depth's mass conserved."""
    N, k = 16, 5
    o, q0, sbar = mountain_case(N, k)
    s = hp.Sphere(N, k)
    q = to_dev(q0)
    s.step(q, 600.0, 1)  # captures a flat step graph for (q, dt)
    q.copy_(to_dev(q0))
    s.set_topography(sbar)
    m0 = s.mass(q)
    s.step(q, 600.0, 5)
    ref = o.step(q0, 600.0, 5)
    got = q.cpu().numpy()
    assert max(rel_l2(got, ref)) < 1e-12, rel_l2(got, ref)
    # the surface really acts: the flat run from the same state differs by percents
    flat = O.Oracle(N, k).step(q0, 600.0, 5)
    assert max(rel_l2(got, flat)) > 1e-6
    assert abs(s.mass(q) - m0) / abs(m0) < 1e-14
    assert s.status() == 0


def test_weno5_steps_over_mountain_fp64(hp):
    """SSP-RK3 steps of section 5.2's flow over the mountain with WENO5 (C16, dt = 600 s):
    states against the oracle at 1e-12, the depth's mass conserved, and the surface acting."""
    N, k = 16, 5
    o, q0, sbar = mountain_case(N, k, scheme=O.WENO)
    s = hp.Sphere(N, k, scheme=hp.HOPE_WENO2D)
    s.set_topography(sbar)
    q = to_dev(q0)
    m0 = s.mass(q)
    s.step(q, 600.0, 5)
    ref = o.step(q0, 600.0, 5)
    got = q.cpu().numpy()
    assert max(rel_l2(got, ref)) < 1e-12, rel_l2(got, ref)
    flat = O.Oracle(N, k, scheme=O.WENO).step(q0, 600.0, 5)
    assert max(rel_l2(got, flat)) > 1e-6
    assert abs(s.mass(q) - m0) / abs(m0) < 1e-14
    assert s.status() == 0


def test_zero_surface_and_removal(hp):
    """A zero surface adds exact zeros (psi_B weights and edge values all 0), so the
    tendency equals the flat one to the last bits; removing the surface restores the flat
    kernels and their result bit for bit."""
    N, k = 12, 5
    o = O.Oracle(N, k)
    q = to_dev(perturb_h(o.rossby_haurwitz(), noise_field((6, N, N), 1)))
    s = hp.Sphere(N, k)
    flat = s.tendency(q).cpu().numpy()
    s.set_topography(np.zeros((6, N, N)))
    zero = s.tendency(q).cpu().numpy()
    assert np.max(np.abs(zero - flat)) <= 1e-15 * np.max(np.abs(flat))
    s.set_topography(None)
    assert s.launches_per_stage() == 4
    assert np.array_equal(s.tendency(q).cpu().numpy(), flat)


@pytest.mark.parametrize("scheme", ["tpp", "weno"])
def test_fp32_tendency_over_mountain(hp, scheme):
    """FP32 context (tables built in FP64, stored in FP32) against the FP64 oracle."""
    N, k = 17, 5
    o, q, sbar = mountain_case(N, k, noise_seed=5, scheme=O.TPP if scheme == "tpp" else O.WENO)
    s = hp.Sphere(N, k, scheme=hp.HOPE_TPP if scheme == "tpp" else hp.HOPE_WENO2D, precision=hp.HOPE_FP32)
    s.set_topography(sbar)
    d = s.tendency(to_dev(q, torch.float32)).double().cpu().numpy()
    err = rel_l2(d, o.tendency(q))
    assert max(err) < 1e-4, err


def test_topography_limits(hp):
    """The dimension-by-dimension comparator and ensembles refuse a surface, a non-finite
    value is an invalid argument, and the adjoint runs with a surface set."""
    import paper_2411_19185_gb300._lib as L
    N, k = 8, 3
    sbar = np.full((6, N, N), 100.0)
    with pytest.raises(L.HopeError) as e:
        hp.Sphere(N, 5, scheme=hp.HOPE_WENO1D).set_topography(np.full((6, N, N), 100.0))
    assert e.value.code == -6
    with pytest.raises(L.HopeError) as e:
        hp.Sphere([N, N], k).set_topography(sbar)
    assert e.value.code == -6
    s = hp.Sphere(N, k)
    bad = sbar.copy()
    bad[0, 0, 0] = np.nan
    with pytest.raises(L.HopeError) as e:
        s.set_topography(bad)
    assert e.value.code == -1
    s.set_topography(sbar)
    q = to_dev(O.Oracle(N, k).geostrophic(u0=U0, phi0=H0 * G))
    assert torch.isfinite(s.tendency_vjp(q, torch.ones_like(q))).all()  # the adjoint covers the surface


# ------------------------------------------------------------------ adjoint over a surface
def _fd_check(s, q, seed, h=1e-6, step_dt=None):
    from synth import fd_direction
    d = torch.from_numpy(fd_direction(q.shape, seed)).cuda() * q.abs().mean(dim=(1, 2, 3), keepdim=True)
    lam = torch.from_numpy(fd_direction(q.shape, seed + 1)).cuda()
    if step_dt is None:
        f = lambda x: s.tendency(x.contiguous())  # noqa: E731
        adj = torch.sum(s.tendency_vjp(q, lam) * d).item()
    else:
        def f(x):
            y = x.contiguous().clone()
            s.step(y, step_dt)
            return y
        adj = torch.sum(s.step_vjp(q, lam, step_dt) * d).item()
    fd = torch.sum(lam * (f(q + h * d) - f(q - h * d))).item() / (2 * h)
    return adj, fd


@pytest.mark.parametrize("k,N", [(3, 10), (5, 12), (7, 14)])
def test_tpp_tendency_vjp_over_mountain_matches_central_differences(hp, k, N):
    """The adjoint of the topography terms (LMARS with phi_t, psi_B's stencil map) with the
    TPP reconstruction: <lam, dL/dq . d> by central differences of the CUDA forward equals
    <(dL/dq)^T lam, d> to 1e-6 over section 5.2's mountain."""
    _, q, sbar = mountain_case(N, k, noise_seed=7)
    s = hp.Sphere(N, k)
    s.set_topography(sbar)
    adj, fd = _fd_check(s, to_dev(q), 61)
    assert abs(adj - fd) <= 1e-6 * abs(fd), (adj, fd)
    assert s.status() == 0


def test_tpp_step_vjp_over_mountain_matches_central_differences(hp):
    """One SSP-RK3 step's adjoint over the mountain (TPP5, C12, dt = 600 s), and the taped
    step adjoint equal to the recomputing one."""
    N, k = 12, 5
    _, q0, sbar = mountain_case(N, k, noise_seed=8)
    s = hp.Sphere(N, k)
    s.set_topography(sbar)
    q = to_dev(q0)
    adj, fd = _fd_check(s, q, 63, step_dt=600.0)
    assert abs(adj - fd) <= 1e-6 * abs(fd), (adj, fd)
    from synth import fd_direction
    lam = torch.from_numpy(fd_direction(q.shape, 65)).cuda()
    tape = torch.empty(s.tape_bytes(), dtype=torch.uint8, device="cuda")
    a = s.step_vjp(q, lam, 600.0)
    qr = q.clone()
    s.step_record(qr, 600.0, tape)
    b = s.step_vjp_tape(q, tape, lam, 600.0)
    assert (torch.linalg.norm(a - b) / torch.linalg.norm(a)).item() < 1e-13
    assert s.status() == 0


@pytest.mark.parametrize("k,N", [(3, 10), (5, 11)])
def test_weno_tendency_vjp_over_mountain_matches_central_differences(hp, k, N):
    """WENO2D over the mountain: the adjoint recomputes its forward on sqrtG phi_t; on a
    rough depth (30% seeded noise, so that no two indicators of a cell are close and tau
    has no kink within the step) central differences agree to 1e-6."""
    o = O.Oracle(N, k, scheme=O.WENO)
    o.set_mountain()
    q = o.geostrophic(u0=U0, phi0=H0 * G)
    q = np.ascontiguousarray(perturb_h(q, noise_field((6, N, N), 9), amp=0.3))
    s = hp.Sphere(N, k, scheme=hp.HOPE_WENO2D)
    s.set_topography(o.topography())
    adj, fd = _fd_check(s, to_dev(q), 67)
    assert abs(adj - fd) <= 1e-6 * abs(fd), (adj, fd)
    assert s.status() == 0
