"""Ensembles at uneven resolutions: one persistent cooperative launch per RK stage (TPP),
checked against independent single-sphere contexts, the oracle, the autotuner and the
bounded grid-barrier timeout."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from synth import noise_field, perturb_h  # noqa: E402


@pytest.fixture(scope="module")
def hp():
    import paper_2411_19185_gb300 as hp
    hp.load()
    return hp


def member_states(members, seed=0, k=3):
    out = []
    for m, N in enumerate(members):
        o = O.Oracle(N, k)
        out.append(perturb_h(o.rossby_haurwitz(), noise_field((6, N, N), seed, member=m)))
    return out


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_ensemble_persistent_matches_single_spheres(hp, prec):
    """Three steps of an uneven ensemble in the persistent launch equal the same steps of
    single-sphere contexts (separate kernels): to 1e-15 in FP64; in FP32 to a few units in
    the last place (the persistent kernel is a different compilation, and the compiler may
    contract a product and a sum into one FMA in one kernel and not in the other)."""
    members = [12, 20, 16, 12]
    P = hp.HOPE_FP64 if prec == "fp64" else hp.HOPE_FP32
    dt = torch.float64 if prec == "fp64" else torch.float32
    ens = hp.Sphere(members, 5, precision=P)
    assert ens.launches_per_stage() == 1
    states = member_states(members, 3)
    q = torch.cat([torch.from_numpy(s).reshape(-1) for s in states]).to("cuda", dt)
    ens.step(q, 600.0, 3)
    for m, N in enumerate(members):
        s = hp.Sphere(N, 5, precision=P)
        qm = torch.from_numpy(states[m]).to("cuda", dt)
        s.step(qm, 600.0, 3)
        a, b = ens.member(q, m).double().cpu().numpy(), qm.double().cpu().numpy()
        tol = 1e-15 if prec == "fp64" else 2.0 ** -21
        assert np.max(np.abs(a - b)) <= tol * np.max(np.abs(b)), (m, np.max(np.abs(a - b)))
    assert ens.status() == 0


def test_ensemble_member_vs_oracle(hp):
    members = [10, 14]
    ens = hp.Sphere(members, 5)
    states = member_states(members, 4)
    q = torch.cat([torch.from_numpy(s).reshape(-1) for s in states]).cuda()
    ens.step(q, 600.0, 2)
    for m, N in enumerate(members):
        ref = O.Oracle(N, 5).step(states[m], 600.0, 2)
        got = ens.member(q, m).cpu().numpy()
        assert max(np.linalg.norm(got[v] - ref[v]) / np.linalg.norm(ref[v]) for v in range(3)) < 1e-12


def test_batching_form_full_size_sample(hp):
    """The full batching workload: 64 members (32 x C48, 24 x C96, 8 x C192), TPP7, FP32,
    Rossby-Haurwitz wave 4 plus 1% seeded h noise per member, dt = 45 s.  Two graph-replayed
    steps of the ensemble equal the same steps of single-sphere contexts for one member of
    each resolution to a few units in the last place; mass per member is conserved to FP32
    round-off."""
    members = [48] * 32 + [96] * 24 + [192] * 8
    ens = hp.Sphere(members, 7, precision=hp.HOPE_FP32)
    q = ens.empty()
    rh = {}
    for N in (48, 96, 192):
        s = hp.Sphere(N, 7, precision=hp.HOPE_FP32)
        rh[N] = (s, s.rossby_haurwitz().double().cpu().numpy())
    for m, N in enumerate(members):
        ens.member(q, m).copy_(torch.from_numpy(perturb_h(rh[N][1], noise_field((6, N, N), 0, member=m))))
    q0 = q.clone()
    m0 = ens.mass(q)
    ens.step(q, 45.0, 2)
    for m in (0, 32, 56):
        N = members[m]
        s = rh[N][0]
        qm = ens.member(q0, m).clone()
        s.step(qm, 45.0, 2)
        a, b = ens.member(q, m).double(), qm.double()
        assert (a - b).abs().max().item() <= 2.0 ** -21 * b.abs().max().item(), m
    m1 = ens.mass(q)
    assert max(abs(a - b) / abs(b) for a, b in zip(m1, m0)) < 2e-7
    assert ens.status() == 0


CANDIDATES = [(16, 8), (8, 16), (32, 4), (16, 4), (12, 10), (24, 5), (8, 8), (16, 16), (32, 8), (16, 12),
              (24, 10), (12, 20)]


def test_autotune_reports_shapes_and_keeps_the_results(hp):
    """The persistent stage's autotuner times every candidate (tile shape x block size) and
    keeps the fastest; a tile shape only regroups cells, so the steps after tuning equal a
    fresh context's (default shape) bitwise, and step graphs captured before the retune are
    dropped rather than replayed with the old shape."""
    members = [16, 24, 13]
    ens = hp.Sphere(members, 7, precision=hp.HOPE_FP32)
    ref = hp.Sphere(members, 7, precision=hp.HOPE_FP32)
    q0 = torch.cat([torch.from_numpy(s).reshape(-1) for s in member_states(members, 2, 7)]).to("cuda", torch.float32)
    qa = q0.clone()
    ens.step(qa, 450.0, 1)  # captures a graph with the initial shape
    ms, shape, grid = ens.autotune(reps=3)
    assert len(ms) >= 8 and all(t > 0 for t in ms), ms
    assert shape in CANDIDATES and grid >= 152
    qc = q0.clone()  # a new buffer: the FP32 low word of qa's earlier step does not carry over
    qb = q0.clone()
    ens.step(qc, 450.0, 2)
    ref.step(qb, 450.0, 2)
    assert torch.equal(qc, qb)
    assert ens.status() == 0


def test_grid_barrier_timeout_is_reported_and_recoverable(hp):
    """The persistent stage's grid barrier waits are bounded: with the test hook, no block
    is released, every block gives up after about a second, the status word reports
    HOPE_STATUS_TIMEOUT and the context keeps working afterwards."""
    members = [8, 10]
    ens = hp.Sphere(members, 3)
    states = member_states(members, 5)
    q = torch.cat([torch.from_numpy(s).reshape(-1) for s in states]).cuda()
    good = ens.tendency(q)
    torch.cuda.synchronize()
    assert ens.status() == 0
    hp._lib.check(hp._lib.load().hope_inject_fault(ens._h, 1))
    ens.tendency(q)
    st = ens.status()
    assert st & hp._lib.HOPE_STATUS_TIMEOUT
    again = ens.tendency(q)
    assert ens.status() == 0
    assert torch.equal(again, good)


def test_persistent_phase_times_are_reported(hp):
    """Profiling of the persistent stage: four positive phase times per stage, and the same
    state as an unprofiled step (the stamps only time the phases)."""
    members = [12, 16, 12]
    ens = hp.Sphere(members, 5, precision=hp.HOPE_FP32)
    states = member_states(members, 9)
    q = torch.cat([torch.from_numpy(s).reshape(-1) for s in states]).to("cuda", torch.float32)
    q2 = q.clone()
    ens.step(q2, 600.0)
    ens.set_profiling(True)
    ens.step(q, 600.0)
    kt = ens.kernel_times()
    ens.set_profiling(False)
    assert len(kt) == 3 and all(len(st) == 4 and all(t > 0 for t in st) for st in kt), kt
    assert torch.equal(q, q2)


# --------------------------------------------------------------- ensemble adjoint
def _ens_state(members, k, seed, dtype=torch.float64):
    return torch.cat([torch.from_numpy(s).reshape(-1) for s in member_states(members, seed, k)]).to("cuda", dtype)


def _dirn(n, seed, dtype=torch.float64):
    from synth import fd_direction
    return torch.from_numpy(fd_direction((n,), seed)).to("cuda", dtype)


@pytest.mark.parametrize("k", [5, 7])
def test_ensemble_tendency_vjp_in_one_launch_equals_single_spheres(hp, k):
    """The stage VJP of an uneven ensemble runs as one persistent launch over all members
    (forward recompute, flux, reconstruction, gather and transposed ghost phases); member by
    member it equals the single-sphere VJP kernels to 1e-13 (FP64)."""
    members = [12, 17, 14]
    ens = hp.Sphere(members, k)
    q = _ens_state(members, k, 21)
    lam = _dirn(q.numel(), 22)
    g = ens.tendency_vjp(q, lam)
    for m, N in enumerate(members):
        s = hp.Sphere(N, k)
        ref = s.tendency_vjp(ens.member(q, m).contiguous(), ens.member(lam, m).contiguous())
        err = (torch.linalg.norm(ens.member(g, m) - ref) / torch.linalg.norm(ref)).item()
        assert err < 1e-13, (m, err)
    assert ens.status() == 0


@pytest.mark.parametrize("rk", ["ssp", "ws"])
def test_ensemble_step_vjp_equals_single_spheres(hp, rk):
    """The step VJP of an ensemble (stage states recomputed by the persistent forward launch,
    three persistent VJP launches) against the members' single-sphere step VJPs."""
    members, k, dt = [10, 14], 5, 600.0
    R = hp.HOPE_SSPRK3 if rk == "ssp" else hp.HOPE_WSRK3
    ens = hp.Sphere(members, k, rk=R)
    q = _ens_state(members, k, 23)
    lam = _dirn(q.numel(), 24)
    g = ens.step_vjp(q, lam, dt)
    for m, N in enumerate(members):
        s = hp.Sphere(N, k, rk=R)
        ref = s.step_vjp(ens.member(q, m).contiguous(), ens.member(lam, m).contiguous(), dt)
        err = (torch.linalg.norm(ens.member(g, m) - ref) / torch.linalg.norm(ref)).item()
        assert err < 1e-13, (m, err)
    assert ens.status() == 0


def test_ensemble_rollout_gradient_equals_members_and_central_differences(hp):
    """Batching form's adjoint (the adjoint of the last steps of an ensemble run): the
    gradient of 0.5 |h_T - h_target|^2 after 8 steps (checkpoints every 3, taped reverse
    sweep read in place by the persistent VJP launch) w.r.t. the ensemble's initial state,
    FP64, TPP7, uneven members: equal to the single-sphere rollout gradients to 1e-13 and to
    central differences to 1e-6."""
    members, k, dt, n = [12, 16, 10], 7, 450.0, 8
    ens = hp.Sphere(members, k)
    q0 = _ens_state(members, k, 25)
    target = _ens_state(members, k, 26)

    def loss_ens(x):
        qT = ens.rollout(x, dt, n, checkpoint_every=3)
        tot = 0.0
        for m in range(len(members)):
            tot = tot + 0.5 * torch.sum((ens.member(qT, m)[0] - ens.member(target, m)[0]) ** 2)
        return tot
    x = q0.clone().requires_grad_(True)
    loss_ens(x).backward()
    g = x.grad
    for m, N in enumerate(members):
        s = hp.Sphere(N, k)
        xm = ens.member(q0, m).contiguous().clone().requires_grad_(True)
        qT = s.rollout(xm, dt, n, checkpoint_every=3)
        (0.5 * torch.sum((qT[0] - ens.member(target, m)[0]) ** 2)).backward()
        err = (torch.linalg.norm(ens.member(g, m) - xm.grad) / torch.linalg.norm(xm.grad)).item()
        assert err < 1e-13, (m, err)
    d = _dirn(q0.numel(), 27)
    for m in range(len(members)):  # scaled per member and variable, as the state is
        ens.member(d, m).mul_(ens.member(q0, m).abs().mean(dim=(1, 2, 3), keepdim=True))
    h = 1e-6
    with torch.no_grad():
        fd = (loss_ens(q0 + h * d) - loss_ens(q0 - h * d)).item() / (2 * h)
    adj = torch.sum(g * d).item()
    assert abs(adj - fd) <= 1e-6 * abs(fd), (adj, fd)
    assert ens.status() == 0


def test_fp32_ensemble_gradient_tracks_fp64(hp):
    """The FP32 ensemble's taped rollout gradient against the FP64 one (4 steps, TPP7):
    relative L2 within 1e-4 (FP32 arithmetic through the forward and reverse sweeps)."""
    members, k, dt, n = [12, 16], 7, 450.0, 4
    grads = []
    for P, dty in ((hp.HOPE_FP64, torch.float64), (hp.HOPE_FP32, torch.float32)):
        ens = hp.Sphere(members, k, precision=P)
        x = _ens_state(members, k, 28, dty).requires_grad_(True)
        w = _dirn(x.numel(), 29, dty)
        (w * ens.rollout(x, dt, n, checkpoint_every=2)).sum().backward()
        grads.append(x.grad.double())
        assert ens.status() == 0
    err = (torch.linalg.norm(grads[1] - grads[0]) / torch.linalg.norm(grads[0])).item()
    assert err < 1e-4, err


def test_vjp_launch_barrier_timeout_is_reported_and_recoverable(hp):
    """The persistent VJP launch uses the same bounded grid barriers: with the test hook no
    block is released, every block gives up after about a second, HOPE_STATUS_TIMEOUT is
    reported, and the next VJP is correct."""
    members = [8, 10]
    ens = hp.Sphere(members, 3)
    q = _ens_state(members, 3, 30)
    lam = _dirn(q.numel(), 31)
    good = ens.tendency_vjp(q, lam).clone()
    assert ens.status() == 0
    hp._lib.check(hp._lib.load().hope_inject_fault(ens._h, 1))
    ens.tendency_vjp(q, lam)
    assert ens.status() & hp._lib.HOPE_STATUS_TIMEOUT
    again = ens.tendency_vjp(q, lam)
    assert ens.status() == 0
    assert torch.equal(again, good)


def test_vjp_phase_times_are_reported(hp):
    """Profiling of the persistent stage VJP: six phase times, the two forward-recompute
    phases positive for a recomputing VJP and zero for a taped one, the rest positive; the
    result equals an unprofiled VJP's."""
    members = [12, 16]
    ens = hp.Sphere(members, 5, precision=hp.HOPE_FP32)
    q = _ens_state(members, 5, 33, torch.float32)
    lam = _dirn(q.numel(), 34, torch.float32)
    ref = ens.tendency_vjp(q, lam).clone()
    ens.set_profiling(True)
    got = ens.tendency_vjp(q, lam)
    t = ens.vjp_phase_times()
    assert len(t) == 6 and all(x > 0 for x in t), t
    tape = torch.empty(ens.tape_bytes(), dtype=torch.uint8, device="cuda")
    qr = q.clone()
    ens.step_record(qr, 450.0, tape)
    ens.step_vjp_tape(q, tape, lam, 450.0)
    t2 = ens.vjp_phase_times()
    ens.set_profiling(False)
    assert t2[0] == 0 and t2[1] == 0 and all(x > 0 for x in t2[2:]), t2
    assert torch.equal(got, ref)
    assert ens.status() == 0
