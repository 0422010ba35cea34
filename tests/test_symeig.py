"""The host eigensolver of the effective matrices (a7) against LAPACK's
(numpy.linalg.eigh): eigenvalues and the leading rows of the eigenvectors,
on random dense, banded (band-Lanczos shaped), degenerate and tiny inputs."""
import numpy as np
import pytest

import paper_2509_22975_gb300 as pkg


@pytest.fixture(scope="module", autouse=True)
def built():
    pkg.build()


def check(A, rows):
    w, X = pkg.mcd_symeig(A, rows)
    wr, Vr = np.linalg.eigh(A)
    scale = max(1.0, np.max(np.abs(wr)))
    assert np.max(np.abs(w - wr)) < 1e-12 * scale * len(A)
    # eigenvectors: compare projectors restricted to the leading rows
    # (columns of a degenerate eigenspace are not unique)
    Pg = X @ X.T
    Pr = Vr[:rows] @ Vr[:rows].T
    assert np.max(np.abs(Pg - Pr)) < 1e-10
    # each computed column is an eigenvector: A V = V w on the full solve
    if rows == len(A):
        assert np.max(np.abs(A @ X - X * w)) < 1e-10 * scale


@pytest.mark.parametrize("n", [1, 2, 3, 17, 120])
def test_random_dense(n):
    rng = np.random.default_rng(n)
    A = rng.normal(size=(n, n))
    check(A + A.T, n)


def test_banded_leading_rows():
    rng = np.random.default_rng(7)
    n, p = 300, 12
    A = np.zeros((n, n))
    for k in range(p + 1):
        d = rng.normal(size=n - k)
        A += np.diag(d, k) + (np.diag(d, -k) if k else 0)
    check(A, p)


def test_degenerate_and_diagonal():
    A = np.diag([3.0, 1.0, 1.0, 1.0, -2.0, 0.0])
    check(A, 6)
    rng = np.random.default_rng(3)
    Qm, _ = np.linalg.qr(rng.normal(size=(40, 40)))
    A = Qm @ np.diag(np.repeat([1.0, 2.0, 5.0, -1.0], 10)) @ Qm.T
    check(0.5 * (A + A.T), 40)
