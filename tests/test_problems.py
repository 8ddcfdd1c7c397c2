"""Pins for the shared input generators (they define the matrices both sides use)."""
import itertools

import numpy as np
import scipy.sparse as sp

import problems as P


def _dense(csr):
    rp, ci, v = csr
    n = len(rp) - 1
    return sp.csr_matrix((v, ci, rp), shape=(n, n)).toarray()


def _lap1d(m):
    return sp.diags([-1.0, 2.0, -1.0], [-1, 0, 1], shape=(m, m))


def test_poisson2d_is_kronecker_sum():
    nx, ny = 5, 3
    K = sp.kron(sp.eye(ny), _lap1d(nx)) + sp.kron(_lap1d(ny), sp.eye(nx))
    assert np.array_equal(_dense(P.poisson_csr((nx, ny))), K.toarray())


def test_poisson3d_is_kronecker_sum():
    nx, ny, nz = 4, 3, 2
    K = (sp.kron(sp.eye(nz * ny), _lap1d(nx))
         + sp.kron(sp.kron(sp.eye(nz), _lap1d(ny)), sp.eye(nx))
         + sp.kron(_lap1d(nz), sp.eye(ny * nx)))
    A = _dense(P.poisson_csr((nx, ny, nz)))
    assert np.array_equal(A, K.toarray())
    rp, ci, v = P.poisson_csr((nx, ny, nz))
    for i in range(len(rp) - 1):
        assert np.all(np.diff(ci[rp[i]:rp[i + 1]]) > 0)


def _brute_varcoef(dims, faces, shift):
    """Assemble sum over faces of c_f (e_a - e_b)(e_a - e_b)^T by loops."""
    if len(dims) == 2:
        nx, ny = dims
        nz = 1
        fx = faces[0].reshape(1, ny, nx + 1)
        fy = faces[1].reshape(1, ny + 1, nx)
        fz = None
    else:
        nx, ny, nz = dims
        fx, fy, fz = faces
    n = nx * ny * nz
    A = np.zeros((n, n))
    idx = lambda x, y, z: x + nx * (y + ny * z)

    def add(a, b, c):
        A[a, a] += c
        if b is not None:
            A[b, b] += c
            A[a, b] -= c
            A[b, a] -= c

    for z, y, x in itertools.product(range(nz), range(ny), range(nx + 1)):
        cells = [idx(x - 1, y, z) if x > 0 else None, idx(x, y, z) if x < nx else None]
        cells = [c for c in cells if c is not None]
        add(cells[0], cells[1] if len(cells) > 1 else None, fx[z, y, x])
    for z, y, x in itertools.product(range(nz), range(ny + 1), range(nx)):
        cells = [idx(x, y - 1, z) if y > 0 else None, idx(x, y, z) if y < ny else None]
        cells = [c for c in cells if c is not None]
        add(cells[0], cells[1] if len(cells) > 1 else None, fy[z, y, x])
    if fz is not None:
        for z, y, x in itertools.product(range(nz + 1), range(ny), range(nx)):
            cells = [idx(x, y, z - 1) if z > 0 else None, idx(x, y, z) if z < nz else None]
            cells = [c for c in cells if c is not None]
            add(cells[0], cells[1] if len(cells) > 1 else None, fz[z, y, x])
    return A + shift * np.eye(n)


def test_varcoef_matches_face_assembly_and_is_spd():
    rng = np.random.default_rng(3)
    for dims in [(4, 3), (3, 3, 2)]:
        faces = P.face_coefficients(dims, 2.0, rng)
        A = _dense(P.stencil_csr(dims, faces, 0.05))
        B = _brute_varcoef(dims, faces, 0.05)
        assert np.allclose(A, B, rtol=1e-14, atol=0)
        assert np.array_equal(A, A.T)
        assert np.linalg.eigvalsh(A).min() > 0
        v = rng.standard_normal(A.shape[0])
        assert np.allclose(P.stencil_apply(dims, v, faces, 0.05), B @ v, rtol=1e-13, atol=1e-13)


def test_constant_faces_equal_poisson():
    dims = (5, 4, 3)
    ones = [np.ones(s) for s in P.face_shapes(dims)]
    assert np.array_equal(_dense(P.stencil_csr(dims, ones)), _dense(P.poisson_csr(dims)))


def test_model_eigenvalues_closed_form():
    lam = P.model_eigenvalues(48, 0.8, 1e3)
    assert lam[0] == 1e-3 and lam[-1] == 1.0
    # i = 2 by hand: lambda_1 + (1/47)(1 - lambda_1) 0.8^46
    assert np.isclose(lam[1], 1e-3 + (1 / 47) * (1 - 1e-3) * 0.8 ** 46, rtol=1e-15)
    assert np.all(np.diff(lam) > 0)


def test_model_problem_structure():
    prob = P.model_problem(48, 0.8, 1e3)
    assert np.allclose(prob.A, prob.A.T)
    assert np.allclose(np.linalg.eigvalsh(prob.A), prob.lam, rtol=1e-10, atol=1e-13)
    assert np.allclose(np.linalg.solve(prob.A, prob.b), 1 / np.sqrt(48), rtol=1e-9)
    Q = P.haar_orthogonal(20, np.random.default_rng(0))
    assert np.allclose(Q.T @ Q, np.eye(20), atol=1e-13)


def test_batch_spec_ranges():
    spec = P.batch_spec(512)
    assert spec.sides.min() >= 32 and spec.sides.max() <= 448
    assert spec.shifts.min() >= 0 and spec.shifts.max() <= 0.1
    assert 3.0e7 < float(np.sum(spec.sides.astype(np.int64) ** 2)) < 4.5e7


def test_generators_are_seeded():
    a = P.poisson2d_64()
    b = P.poisson2d_64()
    assert np.array_equal(a.b, b.b)
    rp, ci, v = a.csr
    assert a.n == 4096 and len(v) == 20224
