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


def test_autotune_reports_shapes(hp):
    ens = hp.Sphere([16, 24], 7, precision=hp.HOPE_FP32)
    ms, shape, grid = ens.autotune(reps=3)
    assert len(ms) == 3 and all(t > 0 for t in ms)
    assert shape in [(16, 8), (16, 4), (32, 4)] and grid >= 152


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
