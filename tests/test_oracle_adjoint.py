"""Pins for the adjoint-gradient oracle: central finite differences of the
loss computed with dense direct solves (numpy.linalg.solve), independent of
any CG code."""
import numpy as np
import scipy.sparse as sp

import oracle as O
import problems as P


def _loss_dense(dims, faces_flat, shift, b, xt):
    shapes = P.face_shapes(dims)
    faces, o = [], 0
    for sh in shapes:
        k = int(np.prod(sh))
        faces.append(faces_flat[o:o + k].reshape(sh))
        o += k
    rp, ci, v = P.stencil_csr(dims, faces, shift)
    n = len(rp) - 1
    A = sp.csr_matrix((v, ci, rp), shape=(n, n)).toarray()
    x = np.linalg.solve(A, b)
    return float(np.sum((x - xt) ** 2))


def test_face_gradient_matches_finite_differences():
    rng = np.random.default_rng(4)
    for dims in [(6, 5), (4, 3, 3)]:
        faces = P.face_coefficients(dims, 1.0, rng)
        ff = P.flat_faces(faces)
        n = int(np.prod(dims))
        b = rng.uniform(-1, 1, n)
        xt = rng.standard_normal(n)
        rp, ci, v = P.stencil_csr(dims, faces, 0.0)
        A = sp.csr_matrix((v, ci, rp), shape=(n, n))
        x, lam = O.adjoint.solve_pair(A, b, lambda x: 2 * (x - xt))
        g = O.adjoint.face_gradient(dims, lam, x)
        h = 1e-6
        for f in rng.choice(len(ff), 12, replace=False):
            e = np.zeros_like(ff)
            e[f] = h * ff[f]
            fd = (_loss_dense(dims, ff + e, 0.0, b, xt) - _loss_dense(dims, ff - e, 0.0, b, xt)) / (2 * e[f])
            assert abs(fd - g[f]) <= 1e-5 * max(abs(fd), 1e-3), (dims, f, fd, g[f])
        # gradient w.r.t. b is lambda
        for i in rng.choice(n, 5, replace=False):
            e = np.zeros(n)
            e[i] = h
            ff0 = ff
            fd = (_loss_dense(dims, ff0, 0.0, b + e, xt) - _loss_dense(dims, ff0, 0.0, b - e, xt)) / (2 * h)
            assert abs(fd - lam[i]) <= 1e-5 * max(abs(fd), 1e-3)


def test_csr_value_gradient_symmetric_direction():
    """Perturbing a_ij and a_ji together keeps A symmetric; the directional
    derivative is the sum of the two entry gradients."""
    rng = np.random.default_rng(5)
    dims = (5, 4)
    rp, ci, v = P.stencil_csr(dims, P.face_coefficients(dims, 1.0, rng), 0.0)
    n = 20
    A = sp.csr_matrix((v, ci, rp), shape=(n, n))
    b = rng.uniform(-1, 1, n)
    xt = rng.standard_normal(n)
    x, lam = O.adjoint.solve_pair(A, b, lambda x: 2 * (x - xt))
    g = O.adjoint.csr_value_gradient(rp, ci, lam, x)
    D = A.toarray()
    rows = np.repeat(np.arange(n), np.diff(rp))
    for e in rng.choice(len(v), 8, replace=False):
        i, j = rows[e], ci[e]
        e2 = np.nonzero((rows == j) & (ci == i))[0][0]
        h = 1e-6
        E = np.zeros((n, n))
        E[i, j] += h
        if e2 != e:
            E[j, i] += h
        lp = np.sum((np.linalg.solve(D + E, b) - xt) ** 2)
        lm = np.sum((np.linalg.solve(D - E, b) - xt) ** 2)
        fd = (lp - lm) / (2 * h)
        ana = g[e] + (g[e2] if e2 != e else 0.0)
        assert abs(fd - ana) <= 1e-5 * max(abs(fd), 1e-3)
