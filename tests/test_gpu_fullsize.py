"""GPU-vs-oracle parity at the sizes and launch configurations that the benchmark times.

Where the oracle cannot evaluate a whole full-size tendency in seconds (C90 WENO9: about
eight minutes on eight cores), it evaluates the same tendency at a sample of cells
(`Oracle.tendency_cells`: the four corners and two edge cells of every panel plus seeded
random cells; only the reconstructions those cells need are computed), and the device's
full-size tendency is compared at those cells.  FP64 bar: relative L2 per variable over
the compared values within 1e-12; adjoints against autograd within 1e-10.
"""
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


def sample_cells(N, n, seed):
    """Corner and edge cells of every panel plus n seeded random cells (flat indices)."""
    rng = np.random.default_rng(seed)
    fixed = [(p * N + j) * N + i for p in range(6)
             for j, i in ((0, 0), (0, N - 1), (N - 1, 0), (N - 1, N - 1), (0, N // 2), (N // 2, N - 1))]
    return np.unique(np.concatenate([np.array(fixed), rng.choice(6 * N * N, size=n, replace=False)]))


def front_cells(q, n, seed):
    """Up to n seeded cells on a discontinuity of q[0] (a cell whose value differs from an
    in-panel neighbour's by more than 1%): where a dam break's tendency is not round-off."""
    a = q[0]
    jump = np.zeros(a.shape, bool)
    dx = np.abs(np.diff(a, axis=2)) > 0.01 * np.abs(a[:, :, 1:])
    dy = np.abs(np.diff(a, axis=1)) > 0.01 * np.abs(a[:, 1:, :])
    jump[:, :, 1:] |= dx
    jump[:, :, :-1] |= dx
    jump[:, 1:, :] |= dy
    jump[:, :-1, :] |= dy
    idx = np.flatnonzero(jump.ravel())
    rng = np.random.default_rng(seed)
    return rng.choice(idx, size=min(n, idx.size), replace=False)


def rel_l2_cols(got, ref):
    return [float(np.linalg.norm(got[v] - ref[v]) / np.linalg.norm(ref[v])) for v in range(3)]


def rh_noise(o, seed):
    return np.ascontiguousarray(perturb_h(o.rossby_haurwitz(), noise_field((6, o.N, o.N), seed)))


@pytest.mark.parametrize("state", ["dam", "rh_noise"])
def test_c90_weno9_fp64_tendency_at_sampled_cells(hp, state):
    """Precision form's FP64 side at full size: C90, WENO9 (the benchmark's context and its
    balanced tile deal), on the 2:1 dam break with Omega = 0 (cells on its front included:
    elsewhere the fluid is at rest and the tendency is round-off) and on the 1%-noise
    Rossby-Haurwitz state; the full-size device tendency at ~300 cells against the oracle's."""
    N, k = 90, 9
    om = 0.0 if state == "dam" else O.OMEGA
    s = hp.Sphere(N, k, hp.HOPE_WENO2D, hp.HOPE_FP64, omega=om, weno_eps=1e-40)
    o = O.Oracle(N, k, scheme=O.WENO, omega=om)
    q = o.dam_break(h_in=10.0, h_out=5.0) if state == "dam" else rh_noise(o, 3)
    d = s.tendency(torch.from_numpy(q).cuda()).cpu().numpy().reshape(3, -1)
    cells = sample_cells(N, 150, 0)
    if state == "dam":  # the fluid at rest has round-off tendencies: sample the front too
        cells = np.unique(np.concatenate([cells, front_cells(q, 150, 1)]))
    ref = o.tendency_cells(q, cells)
    err = rel_l2_cols(d[:, cells], ref)
    assert max(err) < 1e-12, err
    assert s.status() == 0


def test_c180_weno5_fp64_tendency_at_sampled_cells(hp):
    """Differentiation form's forward at full size: C180, WENO5, FP64 (geostrophic flow
    plus the 16 seeded bumps), the device tendency at 200+ cells against the oracle's."""
    from synth import bump_centres
    N, k = 180, 5
    s = hp.Sphere(N, k, hp.HOPE_WENO2D, hp.HOPE_FP64)
    o = O.Oracle(N, k, scheme=O.WENO)
    q = np.ascontiguousarray(perturb_h(o.bumps(bump_centres(16, 0)), noise_field((6, N, N), 19)))
    d = s.tendency(torch.from_numpy(q).cuda()).cpu().numpy().reshape(3, -1)
    cells = sample_cells(N, 200, 1)
    err = rel_l2_cols(d[:, cells], o.tendency_cells(q, cells))
    assert max(err) < 1e-12, err


def test_c180_weno5_fp64_tendency_vjp_matches_autograd_at_full_size(hp):
    """Differentiation form at full size: the hand-written WENO5 tendency VJP of the C180
    context (its own launch shapes) against torch.autograd through the plain PyTorch
    composition of the forward (oracle/torch_ref.py, ~11 s and ~11 GB of host memory),
    relative L2 per variable within 1e-10."""
    from oracle.torch_ref import TorchReference
    from synth import bump_centres
    N, k = 180, 5
    R = TorchReference(N, k, O.WENO)
    s = hp.Sphere(N, k, hp.HOPE_WENO2D, hp.HOPE_FP64)
    q = np.ascontiguousarray(perturb_h(R.o.bumps(bump_centres(16, 0)), noise_field((6, N, N), 23)))
    lam = fd_direction(q.shape, 24)
    qc = torch.from_numpy(q.copy()).requires_grad_(True)
    (R.tendency(qc) * torch.from_numpy(lam)).sum().backward()
    ref = qc.grad.numpy()
    got = s.tendency_vjp(torch.from_numpy(q).cuda(), torch.from_numpy(lam).cuda()).cpu().numpy()
    err = [float(np.linalg.norm(got[v] - ref[v]) / np.linalg.norm(ref[v])) for v in range(3)]
    assert max(err) < 1e-10, err
    assert s.status() == 0


def test_fp64_uneven_ensemble_tpp7_vs_oracle(hp):
    """Batching form's scheme (TPP7) in the persistent launch, FP64, uneven members
    [16, 24, 20] with seeded 1% h noise: two SSP-RK3 steps (dt = 450 s) against the oracle
    member by member, relative L2 within 1e-12."""
    members, k, dt = [16, 24, 20], 7, 450.0
    ens = hp.Sphere(members, k)
    assert ens.launches_per_stage() == 1
    states = [rh_noise(O.Oracle(N, k), 40 + m) for m, N in enumerate(members)]
    q = torch.cat([torch.from_numpy(x).reshape(-1) for x in states]).cuda()
    ens.step(q, dt, 2)
    for m, N in enumerate(members):
        ref = O.Oracle(N, k).step(states[m], dt, 2)
        got = ens.member(q, m).cpu().numpy()
        err = [np.linalg.norm(got[v] - ref[v]) / np.linalg.norm(ref[v]) for v in range(3)]
        assert max(err) < 1e-12, (m, err)
    assert ens.status() == 0


def test_batching_form_full_size_tendency_vs_oracle_at_sampled_cells(hp):
    """The full batching workload's persistent launch (64 members: 32 x C48, 24 x C96,
    8 x C192, TPP7, FP32, Rossby-Haurwitz wave 4 with seeded 1% h noise per member): the
    ensemble tendency of one member of each resolution against the FP64 oracle at sampled
    cells, relative L2 within 1e-4 (the FP32 bound of the tendency tests: unit round-off
    times the ratio of edge fluxes to their divergence on this state)."""
    members = [48] * 32 + [96] * 24 + [192] * 8
    k = 7
    ens = hp.Sphere(members, k, precision=hp.HOPE_FP32)
    q = ens.empty()
    states = {}
    for m, N in enumerate(members):
        if N not in states:
            states[N] = O.Oracle(N, k)
        x = perturb_h(states[N].rossby_haurwitz(), noise_field((6, N, N), 0, member=m))
        ens.member(q, m).copy_(torch.from_numpy(np.ascontiguousarray(x)))
    L = ens.tendency(q)
    for m in (5, 40, 60):
        N = members[m]
        x = ens.member(q, m).double().cpu().numpy()
        cells = sample_cells(N, 120, m)
        ref = states[N].tendency_cells(x, cells)
        got = ens.member(L, m).double().cpu().numpy().reshape(3, -1)[:, cells]
        err = rel_l2_cols(got, ref)
        assert max(err) < 1e-4, (m, err)
    assert ens.status() == 0


@pytest.mark.parametrize("scheme,k,N", [("tpp", 5, 28), ("weno", 5, 24)])
def test_perturbed_jet_steps_vs_oracle(hp, scheme, k, N):
    """Section 5.4's perturbed jet (eqs. 5.16-5.18) as a second workload: five SSP-RK3
    steps of 300 s (the jet sits near the panel-5 boundary) against the oracle, FP64,
    relative L2 within 1e-12; mass conserved to round-off."""
    sch = hp.HOPE_TPP if scheme == "tpp" else hp.HOPE_WENO2D
    s = hp.Sphere(N, k, scheme=sch)
    o = O.Oracle(N, k, scheme=O.TPP if scheme == "tpp" else O.WENO)
    q0 = o.galewsky()
    q = torch.from_numpy(q0).cuda()
    m0 = s.mass(q)
    s.step(q, 300.0, 5)
    ref = o.step(q0, 300.0, 5)
    got = q.cpu().numpy()
    err = [np.linalg.norm(got[v] - ref[v]) / np.linalg.norm(ref[v]) for v in range(3)]
    assert max(err) < 1e-12, err
    assert abs(s.mass(q) - m0) / m0 < 1e-14
    assert s.status() == 0
