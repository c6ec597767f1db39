"""The seeded generators (no GPU): structure of the matrices the tests and the
benchmark share, so that a change of a generator shows up here first."""
import numpy as np

from paper_1806_08020_gb300 import inputs


def _check_csr(A):
    assert A.rowptr[0] == 0 and A.rowptr[-1] == A.colind.size == A.vals.size
    assert np.all(np.diff(A.rowptr) >= 0)
    for i in range(A.n):
        c = A.colind[A.rowptr[i]:A.rowptr[i + 1]]
        assert np.all(np.diff(c) > 0) and (c.size == 0 or (c[0] >= 0 and c[-1] < A.n))


def test_rotation_blocks_structure_and_spectrum():
    """Example 2's stand-in: 2 x 2 blocks [[a, b], [-b, a]] plus a weak coupling
    outside the block; the eigenvalues are a +- i b up to the coupling's size
    (the blocks are normal, so the perturbation is bounded by its norm)."""
    nb = 60
    A = inputs.rotation_blocks(nb, 20.0, 3)
    assert A.n == 2 * nb
    _check_csr(A)
    M = A.to_dense()
    blk = np.zeros_like(M)
    for k in range(nb):
        blk[2 * k:2 * k + 2, 2 * k:2 * k + 2] = M[2 * k:2 * k + 2, 2 * k:2 * k + 2]
        a, b = M[2 * k, 2 * k], M[2 * k, 2 * k + 1]
        assert M[2 * k + 1, 2 * k + 1] == a and M[2 * k + 1, 2 * k] == -b and 0.05 <= a <= 10.0
    E = M - blk
    assert np.count_nonzero(E) <= A.n and np.abs(E).max() < 0.1
    a = np.diag(M)[::2]
    b = np.abs(M[np.arange(0, A.n, 2), np.arange(1, A.n, 2)])
    want = np.concatenate([a + 1j * b, a - 1j * b])
    got = np.linalg.eigvals(M)
    d = np.abs(got[:, None] - want[None, :]).min(axis=1)
    assert d.max() <= np.linalg.norm(E, 2) * 1.001
    # same seed, same matrix; another seed, another one
    B = inputs.rotation_blocks(nb, 20.0, 3)
    assert np.array_equal(A.vals, B.vals) and np.array_equal(A.colind, B.colind)
    assert not np.array_equal(A.vals, inputs.rotation_blocks(nb, 20.0, 4).vals)


def test_stencil_generators_are_valid_csr():
    for A in (inputs.convection_diffusion_2d(7, 30.0), inputs.convection_diffusion_3d(4, 10.0),
              inputs.banded_random(300, 5, 1), inputs.diagonal(np.arange(1.0, 11.0))):
        _check_csr(A)
