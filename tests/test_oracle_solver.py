"""Pins of the oracle's CG and split-Bregman solver on tiny problems, against
dense linear algebra and an independent primal-dual (Chambolle-Pock) solve of
the same objective 1/2 ||P(AX - Y)||^2 + lambda ||W_hp X||_1 (Eqs. 1-5)."""
import numpy as np
import pytest

import oracle
from dense import dense_A, dense_C, dense_W

N8 = 8
V8, B8 = 32, 32   # enough views and bins that A'^T A is well conditioned


def small_geom(filter_=1):
    return oracle.Geometry(n=N8, pixel_mm=1.25, n_views=V8, n_bins=B8, filter=filter_)


@pytest.fixture(scope="module")
def mats():
    g = small_geom()
    A = dense_A(g)
    return {1: (A, dense_C(g)), 0: (A, dense_C(small_geom(0)))}


def smooth_truth():
    y, x = np.mgrid[0:N8, 0:N8] / (N8 - 1.0)
    X = 0.02 * (np.exp(-((x - 0.4) ** 2 + (y - 0.6) ** 2) / 0.08) + (x > 0.7))
    return X


def test_dense_C_matches_oracle_filter(mats):
    g = small_geom()
    _, C = mats[1]
    Y = np.random.Generator(np.random.PCG64(1)).random((V8, B8))
    assert np.allclose(oracle.filter(g, Y).ravel(), C @ Y.ravel(), rtol=0, atol=1e-13)


@pytest.mark.parametrize("filt", [1, 0])
def test_cg_matches_dense_solve(mats, filt):
    g = small_geom(filt)
    A, C = mats[filt]
    mu = 0.05 if filt else 2.0
    M = A.T @ C @ A + mu * np.eye(N8 * N8)
    rhs = np.random.Generator(np.random.PCG64(2)).standard_normal(N8 * N8)
    ref = np.linalg.solve(M, rhs)
    X = oracle.cg(g, rhs.reshape(N8, N8), mu, 64)
    assert np.linalg.norm(X.ravel() - ref) <= 1e-8 * np.linalg.norm(ref)
    # warm start: more steps from the answer keep the answer
    X2 = oracle.cg(g, rhs.reshape(N8, N8), mu, 5, X0=ref.reshape(N8, N8))
    assert np.linalg.norm(X2.ravel() - ref) <= 1e-8 * np.linalg.norm(ref)


def test_cg_stops_on_zero_residual():
    g = small_geom()
    X = oracle.cg(g, np.zeros((N8, N8)), 1.0, 10)
    assert np.all(X == 0.0)


def test_split_bregman_small_lambda_gives_least_squares(mats):
    # lambda -> 0: no shrinkage, so the outer loop is a proximal-point
    # iteration converging to min ||P(AX - Y)||, i.e. A^T C A X = A^T C Y.
    g = small_geom()
    A, C = mats[1]
    Y = (A @ smooth_truth().ravel()).reshape(V8, B8)
    Y += 1e-3 * np.random.Generator(np.random.PCG64(3)).standard_normal(Y.shape)
    ref = np.linalg.solve(A.T @ C @ A, A.T @ C @ Y.ravel())
    X = oracle.solve(g, Y, 0.0, 0.05, 60, 64)
    assert np.linalg.norm(X.ravel() - ref) <= 1e-6 * np.linalg.norm(ref)


def objective(A, C, W, X, Y, lam):
    r = A @ X - Y
    return 0.5 * r @ C @ r + lam * np.abs((W @ X)[N8 * N8:]).sum()


def chambolle_pock(A, C, W, Y, lam, iters=30000):
    """PDHG on min_X G(X) + F(K X), K = high-pass framelet bands (||K|| <= 1),
    G = 1/2 (AX-Y)^T C (AX-Y) (prox by a dense solve), F = lam ||.||_1."""
    K = W[N8 * N8:]
    n = A.shape[1]
    tau = sigma = 0.99
    H = A.T @ C @ A
    Pinv = np.linalg.inv(np.eye(n) + tau * H)
    c = tau * (A.T @ C @ Y)
    x = np.zeros(n)
    xb = x.copy()
    z = np.zeros(K.shape[0])
    for _ in range(iters):
        z = np.clip(z + sigma * (K @ xb), -lam, lam)
        xn = Pinv @ (x - tau * (K.T @ z) + c)
        xb = 2 * xn - x
        x = xn
    return x


@pytest.mark.parametrize("filt", [1, 0])
def test_split_bregman_matches_primal_dual(mats, filt):
    # (filt = 0 is TF-regularised IR, the same solver with C = I)
    g = small_geom(filt)
    A, C = mats[filt]
    W = dense_W(N8)
    Y = A @ smooth_truth().ravel()
    Y += 2e-3 * np.random.Generator(np.random.PCG64(4)).standard_normal(Y.shape)
    lam = 2e-4 if filt else 4e-3
    mu = 2.0 if filt else 30.0      # ADMM penalty near the spectrum of A'^T A
    X, resid = oracle.solve(g, Y.reshape(V8, B8), lam, mu, 1000, 30, return_resid=True)
    Xcp = chambolle_pock(A, C, W, Y, lam)
    f_sb = objective(A, C, W, X.ravel(), Y, lam)
    f_cp = objective(A, C, W, Xcp, Y, lam)
    assert abs(f_sb - f_cp) <= 1e-8 * abs(f_cp)
    # the shrinkage is active (the L1 term matters) ...
    assert np.count_nonzero(np.abs((W @ Xcp)[N8 * N8:]) < 1e-9) > 5
    # ... and the split constraint d = W X is met in the limit
    assert resid[-1] <= 1e-6 * max(resid[0], 1e-30) + 1e-12


# ---------------------------------------------- Eq. (5) and Eq. (6) ----
def test_l2_solve_is_eq5_dense_solution(mats):
    """Enough CG steps solve Eq. (5) exactly: (A^T C A + lam I) X = A^T C Y."""
    g = small_geom()
    A, C = mats[1]
    Y = np.random.Generator(np.random.PCG64(11)).standard_normal((V8, B8))
    lam = 0.3
    ref = np.linalg.solve(A.T @ C @ A + lam * np.eye(N8 * N8), A.T @ C @ Y.ravel())
    X = oracle.l2_solve(g, Y, lam, 200)
    assert np.linalg.norm(X.ravel() - ref) <= 1e-9 * np.linalg.norm(ref)


def test_fbs_without_regulariser_converges_to_least_squares(mats):
    """lam = 0 makes the proximal step the identity (W^T W = I), so Eq. (6)
    is gradient descent on 1/2 ||P(AX - Y)||^2 and converges, for a step below
    2 / ||A^T C A||, to the least-squares solution A^T C A X = A^T C Y."""
    g = small_geom()
    A, C = mats[1]
    M = A.T @ C @ A
    L = np.linalg.eigvalsh(M).max()
    Y = (A @ smooth_truth().ravel()).reshape(V8, B8)
    ref = np.linalg.lstsq(M, A.T @ C @ Y.ravel(), rcond=None)[0]
    X = oracle.fbs(g, Y, 0.0, 1.0 / L, 4000)
    # the component in M's null space stays at its start value, 0, as in lstsq
    assert np.linalg.norm(X.ravel() - ref) <= 1e-6 * np.linalg.norm(ref)


def test_fbs_infinite_threshold_is_the_framelet_lowpass_blur():
    """A threshold above every coefficient zeroes the high-pass bands, so one
    step from X = 0 gives W^T P_0 W X_half with X_half = step A'^T Y: the
    periodic separable blur with (h0 * h0~) = [1, 4, 6, 4, 1] / 16 per axis."""
    g = small_geom()
    Y = np.random.Generator(np.random.PCG64(12)).standard_normal((V8, B8))
    step = 0.7
    X = oracle.fbs(g, Y, 1e30, step, 1)
    Xh = step * oracle.filtered_backproject(g, Y)
    k = np.array([1.0, 4.0, 6.0, 4.0, 1.0]) / 16.0
    blur = sum(k[i] * np.roll(Xh, i - 2, axis=0) for i in range(5))
    blur = sum(k[i] * np.roll(blur, i - 2, axis=1) for i in range(5))
    assert np.allclose(X, blur, rtol=0, atol=1e-12 * np.abs(Xh).max())


def test_fbs_threshold_scales_with_the_step():
    """From X = 0 one iteration is X1 = W^T S_{step lam}(step W A'^T Y)
    = step W^T S_lam(W A'^T Y) (soft thresholding is positively homogeneous),
    so X1 / step does not depend on the step when the threshold is step * lam
    (it would with a threshold of lam alone)."""
    g = small_geom()
    Y = np.random.Generator(np.random.PCG64(13)).standard_normal((V8, B8))
    lam = 0.5 * np.abs(oracle.framelet(oracle.filtered_backproject(g, Y))[1:]).mean()
    a = oracle.fbs(g, Y, lam, 0.5, 1) / 0.5
    b = oracle.fbs(g, Y, lam, 2.0, 1) / 2.0
    assert np.allclose(a, b, rtol=0, atol=1e-12 * np.abs(a).max())
    # and the threshold is active: some but not all high-pass coefficients vanish
    c = oracle.framelet(oracle.filtered_backproject(g, Y))[1:]
    assert 0 < np.count_nonzero(np.abs(c) <= lam) < c.size


# ------------------------------------------ the CG restart between outer steps
def split_bregman_recursive_restart(g, Y, lam, mu, n_outer, n_cg):
    """The split-Bregman loop with each outer step's CG restarted from the
    residual the previous CG left, r + mu (g_new - g_old), instead of the true
    residual rhs - M X that the oracle recomputes (the GPU path's form)."""
    M = lambda x: oracle.filtered_backproject(g, oracle.project(g, x)) + mu * x
    X = np.zeros((g.n, g.n))
    b = np.zeros((9, g.n, g.n))
    gg = np.zeros((g.n, g.n))
    r = oracle.filtered_backproject(g, Y)          # rhs0 - M 0
    for _ in range(n_outer):
        p = r.copy()
        rho = float(np.sum(r * r))
        for _ in range(n_cg):
            if rho == 0.0:
                break
            q = M(p)
            pq = float(np.sum(p * q))
            if not pq > 0.0:
                break
            alpha = rho / pq
            X = X + alpha * p
            r = r - alpha * q
            rho_new = float(np.sum(r * r))
            p = r + (rho_new / rho) * p
            rho = rho_new
        b, g_new, _ = oracle.shrink(X, b, lam / mu)
        r = r + mu * (g_new - gg)                  # rhs changes by mu (g_new - g_old)
        gg = g_new
    return X


@pytest.mark.parametrize("filt", [1, 0])
def test_recursive_cg_restart_is_the_true_residual_restart(filt):
    """CG keeps r = rhs - M X, and between outer steps the right-hand side
    A'^T Y + mu W^T (d - b) changes only by mu (g_new - g_old), so restarting
    from the recursively updated residual is the same algorithm as restarting
    from the true residual (the oracle's form): over 40 outer steps in FP64 the
    two iterates agree to rounding."""
    g = oracle.Geometry(n=16, pixel_mm=1.5, n_views=24, n_bins=40, filter=filt)
    rng = np.random.Generator(np.random.PCG64(21))
    X_true = np.zeros((16, 16))
    X_true[4:12, 5:11] = 0.02
    Y = oracle.project(g, X_true) + 1e-3 * rng.standard_normal((24, 40))
    lam, mu = (3e-4, 1.0) if filt else (3e-3, 20.0)
    ref = oracle.solve(g, Y, lam, mu, 40, 4)
    X = split_bregman_recursive_restart(g, Y, lam, mu, 40, 4)
    assert np.linalg.norm(X - ref) <= 1e-9 * np.linalg.norm(ref)
    # a mistake in the correction (the old g kept) does not agree
    def wrong(g_, Y_, lam_, mu_, n_outer, n_cg):
        Mx = lambda x: oracle.filtered_backproject(g_, oracle.project(g_, x)) + mu_ * x
        X_ = np.zeros((g_.n, g_.n))
        b_ = np.zeros((9, g_.n, g_.n))
        r_ = oracle.filtered_backproject(g_, Y_)
        for _ in range(n_outer):
            p_ = r_.copy()
            rho_ = float(np.sum(r_ * r_))
            for _ in range(n_cg):
                q_ = Mx(p_)
                alpha_ = rho_ / float(np.sum(p_ * q_))
                X_ = X_ + alpha_ * p_
                r_ = r_ - alpha_ * q_
                rn_ = float(np.sum(r_ * r_))
                p_ = r_ + (rn_ / rho_) * p_
                rho_ = rn_
            b_, _, _ = oracle.shrink(X_, b_, lam_ / mu_)
        return X_
    bad = wrong(g, Y, lam, mu, 40, 4)
    assert np.linalg.norm(bad - ref) > 1e-4 * np.linalg.norm(ref)
