"""KL divergence of a block Vecchia approximation from the exact GP (the
fitting measure of the synthetic study of Sec. 7.1, Eq. kldivergence).

For a zero-mean Gaussian p = N(0, Sigma) and the block Vecchia density q built
from the same Sigma (every block conditional p(y_B | y_J) exact),
    KL(p || q) = 1/2 [sum_b log det Sigma_{B|J} - log det Sigma],
and the block terms at y = 0 give sum_b log det Sigma_{B|J} =
-2 l(0) - n log 2 pi.  The pin: on a small problem the identity equals the
textbook Gaussian KL 1/2 [tr(Q Sigma) - n - log det(Q Sigma)] with Q the
precision matrix of q assembled from the conditionals (y_B = A_b y_J + e_b,
e_b ~ N(0, S_b), Q = U^T S^-1 U).
"""
import numpy as np

from oracle import sbv
from synth.inputs import uniform_points


def kl_identity(X, ptr, pts, nbr, cnt, rank, theta, nu2, logdet):
    n = X.shape[0]
    l0 = sbv.loglik(X, np.zeros(n), ptr, pts, nbr, cnt, rank, theta, nu2)
    return -l0 - 0.5 * n * np.log(2 * np.pi) - 0.5 * logdet


def kl_textbook(X, ptr, pts, nbr, cnt, theta, nu2):
    n = X.shape[0]
    idx = np.arange(n)
    Sig = sbv.cov_points(X, idx, idx, theta, nu2)
    U = np.zeros((n, n))
    Sinv = np.zeros((n, n))
    for b in range(len(ptr) - 1):
        B = np.asarray(pts[ptr[b]:ptr[b + 1]])
        J = np.asarray(nbr[b, :cnt[b]])
        U[np.ix_(B, B)] = np.eye(B.size)
        SBB = Sig[np.ix_(B, B)]
        if J.size:
            A = Sig[np.ix_(B, J)] @ np.linalg.inv(Sig[np.ix_(J, J)])
            U[np.ix_(B, J)] = -A
            S = SBB - A @ Sig[np.ix_(J, B)]
        else:
            S = SBB
        Sinv[np.ix_(B, B)] = np.linalg.inv(S)
    Q = U.T @ Sinv @ U
    M = Q @ Sig
    return 0.5 * (np.trace(M) - n - np.linalg.slogdet(M)[1]), np.linalg.slogdet(Sig)[1]


def test_kl_identity_equals_textbook_gaussian_kl():
    n, d = 48, 3
    X = uniform_points(n, d, 5)
    beta = np.array([0.2, 0.5, 1.0])
    theta = np.r_[1.3, 0.01, beta]
    for bc, m in ((48, 5), (8, 6), (6, 0), (1, 0)):
        b = sbv.blocking(X, beta, bc, 3, 7)
        nbr, cnt = sbv.knn(b["Z"], b["blk"], b["rank"], b["centres"], m)
        want, logdet = kl_textbook(X, b["ptr"], b["pts"], nbr, cnt, theta, 5)
        got = kl_identity(X, b["ptr"], b["pts"], nbr, cnt, b["rank"], theta, 5, logdet)
        assert abs(got - want) <= 1e-8 * max(1.0, abs(want)), (bc, m, got, want)
        assert got >= -1e-9
        if bc == 1:            # one block holding every point: q = p
            assert abs(got) <= 1e-9
