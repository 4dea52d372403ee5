"""Hand-written adjoint (vector-Jacobian products) of the stage and of the Runge-Kutta
step, checked against central finite differences of the CUDA forward path (FP64)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from synth import noise_field, perturb_h, fd_direction  # noqa: E402


@pytest.fixture(scope="module")
def hp():
    import paper_2411_19185_gb300 as hp
    hp.load()
    return hp


def state(N, seed=0):
    o = O.Oracle(N, 3)
    q = perturb_h(o.rossby_haurwitz(), noise_field((6, N, N), seed))
    return torch.from_numpy(np.ascontiguousarray(q)).cuda()


def directional(f, q, d, h):
    return (f(q + h * d) - f(q - h * d)) / (2 * h)


@pytest.mark.parametrize("k,N,scheme", [(3, 10, "tpp"), (5, 13, "tpp"), (7, 12, "tpp")])
def test_tendency_vjp_matches_central_differences(hp, k, N, scheme):
    """<lam, dL/dq . d> by central differences (h = 1e-6 |q|) equals <(dL/dq)^T lam, d>
    to a relative 1e-6."""
    s = hp.Sphere(N, k, scheme=hp.HOPE_TPP if scheme == "tpp" else hp.HOPE_WENO2D)
    q = state(N, 1)
    d = torch.from_numpy(fd_direction(q.shape, 2)).cuda() * q.abs().mean(dim=(1, 2, 3), keepdim=True)
    lam = torch.from_numpy(fd_direction(q.shape, 3)).cuda()
    h = 1e-6
    fd = torch.sum(lam * directional(lambda x: s.tendency(x.contiguous()), q, d, h)).item()
    adj = torch.sum(s.tendency_vjp(q, lam) * d).item()
    assert abs(adj - fd) <= 1e-6 * abs(fd), (adj, fd)


@pytest.mark.parametrize("rk", ["ssp", "ws"])
def test_step_vjp_matches_central_differences(hp, rk):
    N, k, dt = 12, 5, 600.0
    s = hp.Sphere(N, k, rk=hp.HOPE_SSPRK3 if rk == "ssp" else hp.HOPE_WSRK3)
    q = state(N, 4)
    d = torch.from_numpy(fd_direction(q.shape, 5)).cuda() * q.abs().mean(dim=(1, 2, 3), keepdim=True)
    lam = torch.from_numpy(fd_direction(q.shape, 6)).cuda()

    def step(x):
        y = x.contiguous().clone()
        s.step(y, dt)
        return y
    h = 1e-6
    fd = torch.sum(lam * directional(step, q, d, h)).item()
    adj = torch.sum(s.step_vjp(q, lam, dt) * d).item()
    assert abs(adj - fd) <= 1e-6 * abs(fd), (adj, fd)


def test_rollout_gradient_with_checkpoints(hp):
    """Gradient of 0.5 |h_T - h_target|^2 after 12 steps (checkpoints every 5) through
    torch.autograd with the hand-written step adjoints, against central differences."""
    N, k, dt, n = 10, 5, 600.0, 12
    s = hp.Sphere(N, k)
    q0 = state(N, 7)
    target = state(N, 8)[0]
    d = torch.from_numpy(fd_direction(q0.shape, 9)).cuda() * q0.abs().mean(dim=(1, 2, 3), keepdim=True)

    def loss(x):
        qT = s.rollout(x, dt, n, checkpoint_every=5)
        return 0.5 * torch.sum((qT[0] - target) ** 2)
    x = q0.clone().requires_grad_(True)
    L0 = loss(x)
    L0.backward()
    g = x.grad
    h = 1e-6
    with torch.no_grad():
        fd = (loss(q0 + h * d) - loss(q0 - h * d)).item() / (2 * h)
    adj = torch.sum(g * d).item()
    assert abs(adj - fd) <= 1e-6 * abs(fd), (adj, fd)


# ------------------------------------------------------------------ WENO adjoint
def smooth_generic_state(N, seed):
    """Rossby-Haurwitz state times (1 + 1e-3 f), f a sum of 12 seeded Gaussian bumps of
    random sign at the cell centres: smooth, and without the wave's exact symmetries."""
    o = O.Oracle(N, 3)
    rng = np.random.default_rng(seed)
    cen = rng.standard_normal((12, 3))
    cen /= np.linalg.norm(cen, axis=1, keepdims=True)
    amp = rng.uniform(-1, 1, 12)
    c = (np.arange(N) + 0.5) * (np.pi / (2 * N)) - np.pi / 4
    f = np.zeros((6, N, N))
    for p in range(6):
        for j in range(N):
            for i in range(N):
                P = O.xyz(p, np.tan(c[i]), np.tan(c[j]))
                f[p, j, i] = np.sum(amp * np.exp(-(np.arccos(np.clip(cen @ P, -1, 1)) / 0.5) ** 2))
    return torch.from_numpy(np.ascontiguousarray(o.rossby_haurwitz() * (1 + 1e-3 * f)[None])).cuda()


@pytest.mark.parametrize("k,N", [(3, 10), (5, 11)])
def test_weno_tendency_vjp_matches_central_differences(hp, k, N):
    """WENO-Z is only piecewise smooth: tau (eq. 3.24) has a kink wherever two indicators
    are equal, and on smooth data the indicators of one cell differ by O(dx) only, so a
    central difference of step h crosses about (pairs x h / dx) kinks -- close to one
    here.  Central differences therefore bound the WENO adjoint only to 1e-4; the exact
    check is the 1e-10 comparison with autograd through the PyTorch reference below.
    The smooth asymmetric state avoids exact ties by symmetry."""
    s = hp.Sphere(N, k, scheme=hp.HOPE_WENO2D)
    q = smooth_generic_state(N, 41)
    d = torch.from_numpy(fd_direction(q.shape, 12)).cuda() * q.abs().mean(dim=(1, 2, 3), keepdim=True)
    lam = torch.from_numpy(fd_direction(q.shape, 13)).cuda()
    h = 1e-6
    fd = torch.sum(lam * directional(lambda x: s.tendency(x.contiguous()), q, d, h)).item()
    adj = torch.sum(s.tendency_vjp(q, lam) * d).item()
    assert abs(adj - fd) <= 1e-4 * abs(fd), (adj, fd)


@pytest.mark.parametrize("k,N", [(3, 10), (5, 11)])
def test_weno_tendency_vjp_matches_central_differences_on_a_rough_state(hp, k, N):
    """Where no two smoothness indicators of a cell are close, tau (eq. 3.24) is smooth
    under the perturbation and central differences bound the WENO adjoint to 1e-6, as for
    TPP: on a rough state (Rossby-Haurwitz times 1 + 0.3 xi, xi ~ U[-1, 1] per cell) the
    indicators of a cell differ by O(beta) while a step of h = 1e-6 |q| moves them by
    O(1e-6 beta), so the difference quotient crosses no kink (on the CPU the same check of
    the PyTorch reference's autograd gradient against the oracle agrees to 2e-9)."""
    s = hp.Sphere(N, k, scheme=hp.HOPE_WENO2D)
    o = O.Oracle(N, 3)
    q = torch.from_numpy(np.ascontiguousarray(
        perturb_h(o.rossby_haurwitz(), noise_field((6, N, N), 51), amp=0.3))).cuda()
    d = torch.from_numpy(fd_direction(q.shape, 52)).cuda() * q.abs().mean(dim=(1, 2, 3), keepdim=True)
    lam = torch.from_numpy(fd_direction(q.shape, 53)).cuda()
    h = 1e-6
    fd = torch.sum(lam * directional(lambda x: s.tendency(x.contiguous()), q, d, h)).item()
    adj = torch.sum(s.tendency_vjp(q, lam) * d).item()
    assert abs(adj - fd) <= 1e-6 * abs(fd), (adj, fd)
    assert s.status() == 0


# ------------------------------------------------------------------ autograd reference
@pytest.mark.parametrize("k,N,scheme", [(3, 8, "tpp"), (5, 10, "tpp"), (3, 8, "weno"), (5, 9, "weno")])
def test_tendency_vjp_matches_torch_autograd_reference(hp, k, N, scheme):
    """(dL/dq)^T lam from the hand-written kernels against torch.autograd through the plain
    PyTorch composition of the forward (oracle/torch_ref.py): relative L2 within 1e-10."""
    from oracle.torch_ref import TorchReference
    sch_o = O.TPP if scheme == "tpp" else O.WENO
    R = TorchReference(N, k, sch_o)
    s = hp.Sphere(N, k, scheme=hp.HOPE_TPP if scheme == "tpp" else hp.HOPE_WENO2D)
    q = state(N, 21)
    lam = torch.from_numpy(fd_direction(q.shape, 22)).cuda()
    qc = q.cpu().clone().requires_grad_(True)
    (R.tendency(qc) * lam.cpu()).sum().backward()
    ref = qc.grad.numpy()
    got = s.tendency_vjp(q, lam).cpu().numpy()
    err = [np.linalg.norm(got[v] - ref[v]) / np.linalg.norm(ref[v]) for v in range(3)]
    assert max(err) < 1e-10, err


def test_rollout_gradient_matches_torch_autograd_reference(hp):
    """Gradient of 0.5 |h_T - h_target|^2 after 4 SSP-RK3 steps w.r.t. the initial state:
    hand-written adjoint with checkpoints against autograd through the PyTorch reference."""
    from oracle.torch_ref import TorchReference
    N, k, dt, n = 8, 3, 600.0, 4
    R = TorchReference(N, k)
    s = hp.Sphere(N, k)
    q0 = state(N, 31)
    target = state(N, 32)[0]
    qc = q0.cpu().clone().requires_grad_(True)
    x = qc
    for _ in range(n):
        x = R.step(x, dt)
    (0.5 * ((x[0] - target.cpu()) ** 2).sum()).backward()
    ref = qc.grad.numpy()
    xg = q0.clone().requires_grad_(True)
    qT = s.rollout(xg, dt, n, checkpoint_every=3)
    (0.5 * ((qT[0] - target) ** 2).sum()).backward()
    got = xg.grad.cpu().numpy()
    err = [np.linalg.norm(got[v] - ref[v]) / np.linalg.norm(ref[v]) for v in range(3)]
    assert max(err) < 1e-10, err


def test_weno_rollout_gradient_matches_torch_autograd_reference(hp):
    """Differentiation form in small: gradient of 0.5 |h_T - h_target|^2 after 3 SSP-RK3
    steps of WENO5 (geostrophic flow plus Gaussian bumps, with 1% seeded h noise) against
    autograd through the PyTorch reference: relative 1e-10.  The noise matters: the zonal
    flow alone ties mirror sub-stencils' indicators exactly, where tau (eq. 3.24) has a kink
    and the gradient is only a subgradient whose pick depends on round-off."""
    from oracle.torch_ref import TorchReference
    from synth import bump_centres
    N, k, dt, n = 9, 5, 900.0, 3
    R = TorchReference(N, k, O.WENO)
    s = hp.Sphere(N, k, scheme=hp.HOPE_WENO2D)
    q0 = torch.from_numpy(np.ascontiguousarray(
        perturb_h(R.o.bumps(bump_centres(16, 0)), noise_field((6, N, N), 17)))).cuda()
    target = torch.from_numpy(np.ascontiguousarray(R.o.bumps(bump_centres(16, 7))))[0].cuda()
    qc = q0.cpu().clone().requires_grad_(True)
    x = qc
    for _ in range(n):
        x = R.step(x, dt)
    (0.5 * ((x[0] - target.cpu()) ** 2).sum()).backward()
    ref = qc.grad.numpy()
    xg = q0.clone().requires_grad_(True)
    qT = s.rollout(xg, dt, n, checkpoint_every=2)
    (0.5 * ((qT[0] - target) ** 2).sum()).backward()
    got = xg.grad.cpu().numpy()
    err = [np.linalg.norm(got[v] - ref[v]) / np.linalg.norm(ref[v]) for v in range(3)]
    assert max(err) < 1e-10, err


@pytest.mark.parametrize("scheme,k,N,rk,prec", [("tpp", 5, 12, "ssp", "fp64"), ("weno", 5, 11, "ssp", "fp64"),
                                                ("tpp", 3, 10, "ws", "fp64"), ("weno", 3, 9, "ssp", "fp32")])
def test_step_vjp_from_tape_equals_recomputing_step_vjp(hp, scheme, k, N, rk, prec):
    """A step recorded with its tape (stage states, ghost rings, edge points) gives the same
    state as hope_step and the same step adjoint as hope_step_vjp, which recomputes the
    stages: the tape only removes forward work (FP64 to 1e-13 relative, FP32 to 1e-5)."""
    P = hp.HOPE_FP64 if prec == "fp64" else hp.HOPE_FP32
    dt_ = torch.float64 if prec == "fp64" else torch.float32
    s = hp.Sphere(N, k, scheme=hp.HOPE_TPP if scheme == "tpp" else hp.HOPE_WENO2D, precision=P,
                  rk=hp.HOPE_SSPRK3 if rk == "ssp" else hp.HOPE_WSRK3)
    q = state(N, 4).to(dt_)
    lam = torch.from_numpy(fd_direction(q.shape, 5)).cuda().to(dt_)
    tape = torch.empty(s.tape_bytes(), dtype=torch.uint8, device="cuda")
    a = s.step_vjp(q, lam, 600.0)
    qr = q.clone()
    s.step_record(qr, 600.0, tape)
    b = s.step_vjp_tape(q, tape, lam, 600.0)
    qs = q.clone()
    s.step(qs, 600.0)
    tol = 1e-13 if prec == "fp64" else 1e-5
    assert (torch.linalg.norm((a - b).double()) / torch.linalg.norm(a.double())).item() < tol
    assert (torch.linalg.norm((qr - qs).double()) / torch.linalg.norm(qs.double())).item() < tol
    assert s.status() == 0


def test_rollout_with_tapes_equals_rollout_with_recompute(hp):
    """The taped backward (each segment recomputed once, step adjoints from tapes) and the
    recomputing backward give the same gradient (FP64, WENO5, 7 steps, checkpoints every 3)."""
    N, k = 10, 5
    s = hp.Sphere(N, k, scheme=hp.HOPE_WENO2D)
    q0 = state(N, 6)
    w = torch.from_numpy(fd_direction(q0.shape, 7)).cuda()
    grads = []
    for tapes in (True, False):
        x = q0.clone().requires_grad_(True)
        qT = s.rollout(x, 600.0, 7, checkpoint_every=3, tapes=tapes)
        (w * qT).sum().backward()
        grads.append(x.grad.clone())
    assert (torch.linalg.norm(grads[0] - grads[1]) / torch.linalg.norm(grads[1])).item() < 1e-13


def test_ssprk3_step_vjp_ignores_the_default_stepper(hp):
    """hope_step_ssprk3_vjp on a Wicker-Skamarock context equals hope_step_vjp on an
    SSP-RK3 context (the same adjoint, bitwise)."""
    N, k = 10, 5
    s_ws = hp.Sphere(N, k, rk=hp.HOPE_WSRK3)
    s_ssp = hp.Sphere(N, k, rk=hp.HOPE_SSPRK3)
    q = state(N, 8)
    lam = torch.from_numpy(fd_direction(q.shape, 9)).cuda()
    assert torch.equal(s_ws.step_ssprk3_vjp(q, lam, 600.0), s_ssp.step_vjp(q, lam, 600.0))
