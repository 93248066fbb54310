"""Property tests of the CPU oracle: unitary invariance of the filter
(Alg. 4) and of the Jacobi eigensolve used by Rayleigh-Ritz (Alg. 2), on
random small cases drawn by hypothesis.  A dropped term, a wrong sign or a
transposed operand in either breaks the invariance for almost every draw.
CPU only."""

import numpy as np
import pytest

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

import oracle  # noqa: E402
from paper_1805_10121_gb300 import synth  # noqa: E402


def _hermitian(n, seed):
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    return (a + a.conj().T) / (2.0 * np.sqrt(n))


@settings(max_examples=25, deadline=None)
@given(n=st.integers(2, 24), b=st.integers(1, 6), seed=st.integers(0, 2**31 - 1),
       degs=st.lists(st.integers(1, 10), min_size=1, max_size=6))
def test_filter_unitary_invariance(n, b, seed, degs):
    """p(U H U^H) U V = U p(H) V: the filter commutes with a change of basis."""
    m = sorted(2 * d for d in (degs * b)[:b])
    H = _hermitian(n, seed)
    lam = np.linalg.eigvalsh(H)
    b_sup = lam[-1] + 0.05
    mu1 = lam[0]
    mu_nn = lam[0] + 0.6 * (lam[-1] - lam[0])
    V = synth.gaussian_block(n, b, seed % 1000).numpy()
    U = synth.unitary_qr(n, seed % 997 + 1).numpy()
    base = oracle.cheb_filter(H, V, m, b_sup, mu1, mu_nn)
    rot = oracle.cheb_filter(U @ H @ U.conj().T, U @ V, m, b_sup, mu1, mu_nn)
    ref = U @ base
    assert np.linalg.norm(rot - ref) <= 1e-10 * max(1.0, np.linalg.norm(ref))


@settings(max_examples=25, deadline=None)
@given(n=st.integers(1, 20), seed=st.integers(0, 2**31 - 1))
def test_jacobi_unitary_invariance(n, seed):
    """eig(U G U^H) = eig(G), and the eigenvectors rotate with U."""
    G = _hermitian(n, seed)
    U = synth.unitary_qr(n, seed % 991 + 1).numpy()
    w0, Z0 = oracle.jacobi_eigh(G)
    w1, Z1 = oracle.jacobi_eigh(U @ G @ U.conj().T)
    scale = max(1.0, np.abs(w0).max())
    assert np.max(np.abs(w1 - w0)) <= 1e-12 * scale
    # each rotated eigenvector is an eigenvector of the rotated matrix
    Gr = U @ G @ U.conj().T
    assert np.linalg.norm(Gr @ (U @ Z0) - (U @ Z0) * w0[None, :]) <= 1e-11 * scale * n


@settings(max_examples=20, deadline=None)
@given(n=st.integers(4, 30), k=st.integers(1, 4), seed=st.integers(0, 2**31 - 1))
def test_householder_qr_span_and_unitarity(n, k, seed):
    """Q has orthonormal columns, R is upper triangular and Q R = X."""
    X = synth.gaussian_block(n, k, seed % 1000).numpy()
    Q, R = oracle.householder_qr(X)
    assert np.linalg.norm(Q.conj().T @ Q - np.eye(k)) < 1e-13
    assert np.linalg.norm(np.tril(R, -1)) == 0.0
    assert np.linalg.norm(Q @ R - X) < 1e-13 * np.linalg.norm(X)
