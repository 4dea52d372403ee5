"""The dimension-by-dimension WENO-Z comparator of section 5.5 (HOPE_WENO1D, reading c31 of
the oracle) on the GPU against the oracle's WENO1D form: tendencies and steps in FP64 at
relative L2 1e-12, the FP32 path at the FP32 tendency bound, and the full-size C90 launch
at sampled cells."""
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


def rh_noise(o, seed):
    return np.ascontiguousarray(perturb_h(o.rossby_haurwitz(), noise_field((6, o.N, o.N), seed)))


def check(d, ref, tol):
    for v in range(3):
        nr = np.linalg.norm(ref[v])
        err = np.linalg.norm(d[v] - ref[v])
        assert err <= tol * max(nr, 1e-12 * np.linalg.norm(ref[0])), (v, err, nr)


@pytest.mark.parametrize("N", [13, 17, 24])
@pytest.mark.parametrize("state", ["rh_noise", "dam"])
def test_tendency_weno1d_fp64(hp, N, state):
    """Tendency (eq. 3.1) with the comparator's reconstruction, FP64, tiles with ragged
    tails: smooth (1%-noise Rossby-Haurwitz) and discontinuous (2:1 dam break) states."""
    s = hp.Sphere(N, 5, scheme=hp.HOPE_WENO1D)
    o = O.Oracle(N, 5, scheme=O.WENO1D)
    q = rh_noise(o, 3) if state == "rh_noise" else o.dam_break(h_in=10.0, h_out=5.0)
    d = s.tendency(torch.from_numpy(q).cuda()).cpu().numpy()
    check(d, o.tendency(q), 1e-12)
    assert s.status() == 0


def test_weno1d_dam_break_steps_fp64(hp):
    """Four SSP-RK3 steps of 300 s of the 2:1 dam break (Omega = 0) with the comparator:
    state against the oracle at 1e-12, mass conserved to round-off."""
    N = 16
    s = hp.Sphere(N, 5, scheme=hp.HOPE_WENO1D, omega=0.0)
    o = O.Oracle(N, 5, scheme=O.WENO1D, omega=0.0)
    q0 = o.dam_break(h_in=10.0, h_out=5.0)
    q = torch.from_numpy(q0).cuda()
    m0 = s.mass(q)
    s.step(q, 300.0, 4)
    check(q.cpu().numpy(), o.step(q0, 300.0, 4), 1e-12)
    assert abs(s.mass(q) - m0) / m0 < 1e-14
    assert s.status() == 0


def test_weno1d_fp32_tendency_vs_oracle(hp):
    """FP32 comparator tendency against the FP64 oracle within the FP32 tendency bound
    (1e-4 relative L2, as for the other schemes on this state)."""
    N = 17
    s = hp.Sphere(N, 5, scheme=hp.HOPE_WENO1D, precision=hp.HOPE_FP32)
    o = O.Oracle(N, 5, scheme=O.WENO1D)
    q = rh_noise(o, 5)
    d = s.tendency(torch.from_numpy(q).cuda().float()).double().cpu().numpy()
    ref = o.tendency(q)
    err = [np.linalg.norm(d[v] - ref[v]) / np.linalg.norm(ref[v]) for v in range(3)]
    assert max(err) < 1e-4, err


def test_weno1d_c90_full_size_at_sampled_cells(hp):
    """The C90 dam-break launch of the anisotropy comparison, FP64: the full-size tendency
    at sampled cells (corners, cube edges, seeded random cells and cells on the front, where
    the tendency is not round-off) against the oracle's."""
    N = 90
    s = hp.Sphere(N, 5, scheme=hp.HOPE_WENO1D, omega=0.0)
    o = O.Oracle(N, 5, scheme=O.WENO1D, omega=0.0)
    q = o.dam_break(h_in=10.0, h_out=5.0)
    d = s.tendency(torch.from_numpy(q).cuda()).cpu().numpy().reshape(3, -1)
    from test_gpu_fullsize import sample_cells, front_cells
    cells = np.unique(np.concatenate([sample_cells(N, 150, 0), front_cells(q, 150, 1)]))
    ref = o.tendency_cells(q, cells)
    check(d[:, cells], ref, 1e-12)


def test_weno1d_has_no_adjoint(hp):
    s = hp.Sphere(8, 5, scheme=hp.HOPE_WENO1D)
    q = s.rossby_haurwitz()
    with pytest.raises(hp.HopeError) as e:
        s.tendency_vjp(q, q.clone())
    assert e.value.code == -6
