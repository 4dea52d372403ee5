"""The PyTorch reference composition (oracle/torch_ref.py, test infrastructure for the
adjoint checks) reproduces the C oracle's forward before its autograd gradient is used."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from oracle.torch_ref import TorchReference
from synth import noise_field, perturb_h


@pytest.mark.parametrize("N,k,scheme,tol", [(8, 3, O.TPP, 1e-13), (10, 5, O.TPP, 1e-13),
                                            (9, 5, O.WENO, 5e-12), (8, 3, O.WENO, 5e-12)])
def test_torch_reference_matches_oracle_tendency(N, k, scheme, tol):
    R = TorchReference(N, k, scheme)
    q = np.ascontiguousarray(perturb_h(R.o.rossby_haurwitz(), noise_field((6, N, N), 1)))
    d_o = R.o.tendency(q)
    d_t = R.tendency(torch.tensor(q)).detach().numpy()
    err = [np.linalg.norm(d_t[v] - d_o[v]) / np.linalg.norm(d_o[v]) for v in range(3)]
    assert max(err) < tol, err


def test_torch_reference_step_matches_oracle():
    N, k = 8, 3
    R = TorchReference(N, k)
    q = np.ascontiguousarray(perturb_h(R.o.rossby_haurwitz(), noise_field((6, N, N), 2)))
    a = R.step(torch.tensor(q), 600.0).detach().numpy()
    b = R.o.step(q, 600.0, 1)
    assert max(np.linalg.norm(a[v] - b[v]) / np.linalg.norm(b[v]) for v in range(3)) < 1e-14
