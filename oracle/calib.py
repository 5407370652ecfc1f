"""Oracle: redundant-baseline calibration of one channel, in FP64 numpy.

TEST INFRASTRUCTURE ONLY: the library's product path never imports this
module, and this module imports nothing from the library.

Paper basis:
  * the system of equations V_ij = g_i g_j^* V_alpha + n_ij (Sec. 2,
    Eq. redcal), solved per channel (footnote to Eq. redcal);
  * logarithmic linearisation (Eq. logcal) -- used here only to start the
    iteration and to evaluate Eq. gaincov;
  * lincal: Taylor expansion of the variables about a starting point
    (Sec. 2, after Eq. logcal) -- a Gauss-Newton solve of chi^2;
  * omnical with damping 0.3 and convergence criterion 1e-10 (Sec. 3);
  * degeneracies: overall amplitude, overall phase, x and y phase slopes
    (Sec. 5.2); the paper fixes them against the simulated gains (Sec. 3);
  * chi^2_r and DoF (Eq. redchi, Eq. dof); uniform noise weights
    (Eq. noisecov);
  * gain covariance (Eq. cov, Eq. gaincov).

Readings where the paper is silent (stated in the design notes): the omnical
update is the simultaneous least-squares fixed point of each variable with
the others held, damped as x <- (1 - 0.3) x + 0.3 x_new, stopped when
|x_new - x| / |x| < tol; lincal is Gauss-Newton on (Re, Im) of every gain and
model visibility with a vanishing Levenberg term (1e-12 of the largest
diagonal) so that the exact degeneracies stay out of each step; the phase
start is a spanning tree over the (1,0) and (0,1) types followed by a
wrapped-residual phase logcal; the output convention is mean ln|g| = 0,
arg g_0 = 0 and arg V_(1,0) = arg V_(0,1) = 0.
"""
from __future__ import annotations

import numpy as np


# --------------------------------------------------------------------------- model
def model(g, V, pi, pj, alpha):
    """m_p = g_i conj(g_j) V_alpha (Eq. redcal without noise)."""
    return g[pi] * np.conj(g[pj]) * V[alpha]


def chi2(vobs, g, V, pi, pj, alpha, w=None):
    """sum_p w_p |V_p - g_i g_j^* V_alpha|^2 (numerator of Eq. redchi)."""
    r = vobs - model(g, V, pi, pj, alpha)
    ww = 1.0 if w is None else w
    return float(np.sum(ww * (r.real ** 2 + r.imag ** 2)))


def chi2_grad(vobs, g, V, pi, pj, alpha, w=None):
    """Gradient of chi^2 as d/dRe + i d/dIm, for gains and model visibilities.

    With r_p = V_p - g_i g_j^* V_a:
      dchi2/dg_k   = -2 [ sum_{p: i_p=k} w r g_j conj(V_a)
                          + sum_{p: j_p=k} w conj(r) g_i V_a ]
      dchi2/dV_a   = -2 sum_{p in a} w r conj(g_i) g_j
    """
    r = vobs - model(g, V, pi, pj, alpha)
    ww = np.ones(len(r)) if w is None else w
    dg = np.zeros(len(g), np.complex128)
    dV = np.zeros(len(V), np.complex128)
    np.add.at(dg, pi, -2.0 * ww * r * g[pj] * np.conj(V[alpha]))
    np.add.at(dg, pj, -2.0 * ww * np.conj(r) * g[pi] * V[alpha])
    np.add.at(dV, alpha, -2.0 * ww * r * np.conj(g[pi]) * g[pj])
    return dg, dV


def dof(P, N, n_ubl):
    """Eq. dof: N_obs - N - N_ubl + 2 (complex units)."""
    return P - N - n_ubl + 2


def chi2_r(vobs, g, V, pi, pj, alpha, sigma2):
    """Eq. redchi with per-pair noise variance sigma2."""
    r = vobs - model(g, V, pi, pj, alpha)
    return float(np.sum((r.real ** 2 + r.imag ** 2) / sigma2)) / dof(len(vobs), len(g), len(V))


# --------------------------------------------------------------------------- degeneracies
def _axis_types(types):
    return types.index((1, 0)), types.index((0, 1))


def _pos(L, N):
    """Lattice coordinates [N, 2] of the antennas: the L x L grid (i = y L + x)
    when L is an int, else L itself -- an [N, 2] array of lattice coordinates
    for arrays that do not fill a square grid (e.g. hexagonal ones, Sec. 3);
    every degeneracy and convention below is linear in these coordinates."""
    if isinstance(L, (int, np.integer)):
        return np.stack([np.arange(L * L) % L, np.arange(L * L) // L], 1).astype(float)
    p = np.asarray(L, float)
    assert p.shape == (N, 2)
    return p


def project(g, V, types, L):
    """Fix the four degeneracies (Sec. 5.2) to the output convention."""
    g = np.asarray(g, np.complex128).copy()
    V = np.asarray(V, np.complex128).copy()
    # amplitude: g -> g / s, V -> V s^2 leaves g_i g_j^* V unchanged
    s = np.exp(np.mean(np.log(np.abs(g))))
    g /= s
    V *= s * s
    # phase slopes: g_i -> g_i e^{i k.r_i}, V_a -> V_a e^{-i k.d_a}
    ax, ay = _axis_types(types)
    k = np.array([np.angle(V[ax]), np.angle(V[ay])])
    pos = _pos(L, len(g))
    g *= np.exp(1j * pos @ k)
    d = np.asarray(types, float)
    V *= np.exp(-1j * d @ k)
    # overall phase
    g *= np.exp(-1j * np.angle(g[0]))
    return g, V


def fit_degeneracies(g_est, g_true, L):
    """Transform g_est by the degeneracies to best match g_true (Sec. 3).

    Wrap-free: q = g_true / g_est; amplitude = exp(mean ln|q|); slopes from
    the mean neighbour phase increments of q; offset from the residual mean.
    """
    q = g_true / g_est
    amp = np.exp(np.mean(np.log(np.abs(q))))
    if isinstance(L, (int, np.integer)):
        qq = q.reshape(L, L)
        kx = np.angle(np.sum(qq[:, 1:] * np.conj(qq[:, :-1]))) if L > 1 else 0.0
        ky = np.angle(np.sum(qq[1:, :] * np.conj(qq[:-1, :]))) if L > 1 else 0.0
    else:   # mean increments over the antenna pairs one lattice step apart
        pos = _pos(L, len(q))
        at = {(int(a), int(b)): n for n, (a, b) in enumerate(pos)}
        sx = sum(q[at[(a + 1, b)]] * np.conj(q[n]) for (a, b), n in at.items() if (a + 1, b) in at)
        sy = sum(q[at[(a, b + 1)]] * np.conj(q[n]) for (a, b), n in at.items() if (a, b + 1) in at)
        kx, ky = float(np.angle(sx)), float(np.angle(sy))
    pos = _pos(L, len(q))
    ramp = np.exp(1j * (pos @ np.array([kx, ky])))
    phi0 = np.angle(np.sum(q * np.conj(ramp)))
    return g_est * amp * ramp * np.exp(1j * phi0)


# --------------------------------------------------------------------------- start point
def _lstsq_rows(n_var, rows_idx, rows_val, rhs, sparse=False):
    """Minimum-norm least-squares solution of the rows given by (index,
    value) lists: numpy's dense solver, or (sparse) LSQR started from zero,
    which converges to the same minimum-norm solution."""
    if not sparse:
        A = np.zeros((len(rhs), n_var))
        for r, (idx, val) in enumerate(zip(rows_idx, rows_val)):
            for c, v in zip(idx, val):
                A[r, c] += v
        sol, *_ = np.linalg.lstsq(A, rhs, rcond=None)
        return sol
    from scipy.sparse import coo_matrix
    from scipy.sparse.linalg import lsqr
    rr, cc, vv = [], [], []
    for r, (idx, val) in enumerate(zip(rows_idx, rows_val)):
        for c, v in zip(idx, val):
            rr.append(r)
            cc.append(c)
            vv.append(v)
    A = coo_matrix((vv, (rr, cc)), shape=(len(rhs), n_var)).tocsr()
    return lsqr(A, rhs, atol=1e-15, btol=1e-15, conlim=1e15, iter_lim=50 * n_var)[0]


def initial_solution(vobs, pi, pj, alpha, types, L, sparse=False):
    """Phase tree + wrapped phase logcal + amplitude logcal (Eq. logcal)."""
    nu = len(types)
    ax, ay = _axis_types(types)
    lookup = {}
    for p in range(len(vobs)):
        if alpha[p] in (ax, ay):
            lookup[(int(pi[p]), int(pj[p]))] = vobs[p]
    if isinstance(L, (int, np.integer)):
        N = L * L
        phi = np.zeros(N)
        for x in range(1, L):                       # along the first row
            phi[x] = phi[x - 1] + np.angle(lookup[(x, x - 1)])
        for y in range(1, L):                       # up every column
            for x in range(L):
                i, j = y * L + x, (y - 1) * L + x
                phi[i] = phi[j] + np.angle(lookup[(i, j)])
    else:
        # breadth-first tree over the axis-type pairs from antenna 0:
        # phi_i - phi_j = arg V_p for p = (i, j) (arg V of both axis types is 0)
        N = len(L)
        phi = np.zeros(N)
        nbrs = [[] for _ in range(N)]
        for (i, j), vp in lookup.items():
            nbrs[j].append((i, np.angle(vp)))
            nbrs[i].append((j, -np.angle(vp)))
        seen = np.zeros(N, bool)
        seen[0] = True
        queue = [0]
        for a in queue:
            for b, dphi in nbrs[a]:
                if not seen[b]:
                    seen[b] = True
                    phi[b] = phi[a] + dphi
                    queue.append(b)
        assert seen.all(), "the axis types do not connect the array"
    # wrapped residual phase logcal: dphi_i - dphi_j + theta_a = wrap(arg V - phi_i + phi_j).
    # Eq. logcal's phase equation holds modulo 2 pi; the branch is taken per
    # redundant group around the group's circular mean, so that a group whose
    # residual phase sits near +-pi does not split across the cut
    res = np.angle(vobs * np.exp(-1j * (phi[pi] - phi[pj])))
    mu = np.zeros(nu, np.complex128)
    np.add.at(mu, alpha, np.exp(1j * res))
    mu = np.angle(mu)
    res = mu[alpha] + np.angle(np.exp(1j * (res - mu[alpha])))
    idx = [(int(pi[p]), int(pj[p]), N + int(alpha[p])) for p in range(len(vobs))]
    sol = _lstsq_rows(N + nu, idx, [(1.0, -1.0, 1.0)] * len(vobs), res, sparse)
    phi = phi + sol[:N]
    # amplitude logcal: eta_i + eta_j + a_alpha = ln|V_p|
    sol = _lstsq_rows(N + nu, idx, [(1.0, 1.0, 1.0)] * len(vobs), np.log(np.abs(vobs)), sparse)
    g = np.exp(sol[:N] + 1j * phi)
    V = np.zeros(nu, np.complex128)
    cnt = np.zeros(nu)
    np.add.at(V, alpha, vobs / (g[pi] * np.conj(g[pj])))
    np.add.at(cnt, alpha, 1.0)
    return g, V / cnt


# --------------------------------------------------------------------------- solvers
def _jacobian(g, V, pi, pj, alpha):
    """Real Jacobian of [Re m; Im m] w.r.t. x = [Re g, Im g, Re V, Im V]."""
    N, nu, P = len(g), len(V), len(pi)
    J = np.zeros((2 * P, 2 * N + 2 * nu))
    rows = np.arange(P)
    dgi = np.conj(g[pj]) * V[alpha]          # dm/dRe g_i ; dm/dIm g_i = i*dgi
    dgj = g[pi] * V[alpha]                   # dm/dRe g_j ; dm/dIm g_j = -i*dgj
    dv = g[pi] * np.conj(g[pj])              # dm/dRe V   ; dm/dIm V = i*dv
    # Re g_i
    np.add.at(J, (rows, pi), dgi.real)
    np.add.at(J, (P + rows, pi), dgi.imag)
    # Im g_i
    np.add.at(J, (rows, N + pi), -dgi.imag)
    np.add.at(J, (P + rows, N + pi), dgi.real)
    # Re g_j
    np.add.at(J, (rows, pj), dgj.real)
    np.add.at(J, (P + rows, pj), dgj.imag)
    # Im g_j: -i*dgj
    np.add.at(J, (rows, N + pj), dgj.imag)
    np.add.at(J, (P + rows, N + pj), -dgj.real)
    # Re V
    np.add.at(J, (rows, 2 * N + alpha), dv.real)
    np.add.at(J, (P + rows, 2 * N + alpha), dv.imag)
    # Im V
    np.add.at(J, (rows, 2 * N + nu + alpha), -dv.imag)
    np.add.at(J, (P + rows, 2 * N + nu + alpha), dv.real)
    return J


def _jacobian_sparse(g, V, pi, pj, alpha):
    """The Jacobian of _jacobian as a scipy sparse matrix (same entries,
    duplicates summed) for arrays too large for the dense form."""
    from scipy.sparse import coo_matrix
    N, nu, P = len(g), len(V), len(pi)
    rows = np.arange(P)
    dgi = np.conj(g[pj]) * V[alpha]
    dgj = g[pi] * V[alpha]
    dv = g[pi] * np.conj(g[pj])
    R, Cc, X = [], [], []

    def put(r, c, v):
        R.append(r)
        Cc.append(c)
        X.append(v)
    put(rows, pi, dgi.real)
    put(P + rows, pi, dgi.imag)
    put(rows, N + pi, -dgi.imag)
    put(P + rows, N + pi, dgi.real)
    put(rows, pj, dgj.real)
    put(P + rows, pj, dgj.imag)
    put(rows, N + pj, dgj.imag)
    put(P + rows, N + pj, -dgj.real)
    put(rows, 2 * N + alpha, dv.real)
    put(P + rows, 2 * N + alpha, dv.imag)
    put(rows, 2 * N + nu + alpha, -dv.imag)
    put(P + rows, 2 * N + nu + alpha, dv.real)
    return coo_matrix((np.concatenate(X), (np.concatenate(R), np.concatenate(Cc))),
                      shape=(2 * P, 2 * N + 2 * nu)).tocsr()


def _degenerate_directions(g, V, types_d, L):
    """Real tangent vectors of the four degeneracies at (g, V), in the
    ordering x = [Re g, Im g, Re V, Im V]: amplitude (g, -2V), phase (i g, 0)
    and the two slopes (i x_i g_i, -i dx_a V_a), (i y_i g_i, -i dy_a V_a)."""
    N = len(g)
    pos = _pos(L, N)
    xs, ys = pos[:, 0], pos[:, 1]
    dirs = [(g, -2.0 * V), (1j * g, 0.0 * V),
            (1j * xs * g, -1j * types_d[:, 0] * V), (1j * ys * g, -1j * types_d[:, 1] * V)]
    return np.stack([np.concatenate([a.real, a.imag, b.real, b.imag]) for a, b in dirs], 1)


def lincal(vobs, pi, pj, alpha, g, V, types, L, tol=1e-10, maxiter=200, sparse=False):
    """Gauss-Newton on chi^2 about the current point (Sec. 2, lincal).
    sparse: the same normal equations in scipy sparse form, solved by a
    sparse direct factorisation (for arrays too large for the dense form)."""
    types_d = np.asarray(types, float)
    g = np.asarray(g, np.complex128).copy()
    V = np.asarray(V, np.complex128).copy()
    N, nu = len(g), len(V)
    for it in range(1, maxiter + 1):
        r = vobs - model(g, V, pi, pj, alpha)
        if sparse:
            from scipy.sparse import identity
            from scipy.sparse.linalg import spsolve
            J = _jacobian_sparse(g, V, pi, pj, alpha)
            A = (J.T @ J).tocsc()
            b = J.T @ np.concatenate([r.real, r.imag])
            A = A + (1e-12 * A.diagonal().max()) * identity(A.shape[0], format="csc")
            delta = spsolve(A, b)
        else:
            J = _jacobian(g, V, pi, pj, alpha)
            A = J.T @ J
            b = J.T @ np.concatenate([r.real, r.imag])
            A[np.diag_indices_from(A)] += 1e-12 * np.max(np.diag(A))
            c = np.linalg.cholesky(A)
            delta = np.linalg.solve(c.T, np.linalg.solve(c, b))
        # keep the four exact degeneracies (Sec. 5.2) out of the step
        Q, _ = np.linalg.qr(_degenerate_directions(g, V, types_d, L))
        delta -= Q @ (Q.T @ delta)
        x = np.concatenate([g.real, g.imag, V.real, V.imag])
        g = g + delta[:N] + 1j * delta[N:2 * N]
        V = V + delta[2 * N:2 * N + nu] + 1j * delta[2 * N + nu:]
        if np.linalg.norm(delta) <= tol * np.linalg.norm(x):
            return g, V, it, True
    return g, V, maxiter, False


def omnical(vobs, pi, pj, alpha, g, V, damping=0.3, tol=1e-10, maxiter=100000):
    """Damped simultaneous least-squares fixed point (omnical, Sec. 3)."""
    g = np.asarray(g, np.complex128).copy()
    V = np.asarray(V, np.complex128).copy()
    N, nu = len(g), len(V)
    for it in range(1, maxiter + 1):
        zi = np.conj(g[pj]) * V[alpha]           # coefficient of g_i in m_p
        zj = g[pi] * V[alpha]                    # coefficient of conj(g_j)
        num = np.zeros(N, np.complex128)
        den = np.zeros(N)
        np.add.at(num, pi, vobs * np.conj(zi))
        np.add.at(den, pi, np.abs(zi) ** 2)
        np.add.at(num, pj, np.conj(vobs) * zj)
        np.add.at(den, pj, np.abs(zj) ** 2)
        g_new = num / den
        zv = g[pi] * np.conj(g[pj])
        vn = np.zeros(nu, np.complex128)
        vd = np.zeros(nu)
        np.add.at(vn, alpha, vobs * np.conj(zv))
        np.add.at(vd, alpha, np.abs(zv) ** 2)
        V_new = vn / vd
        x = np.concatenate([g, V])
        xn = np.concatenate([g_new, V_new])
        change = np.linalg.norm(xn - x) / np.linalg.norm(x)
        g = (1.0 - damping) * g + damping * g_new
        V = (1.0 - damping) * V + damping * V_new
        if change < tol:
            return g, V, it, True
    return g, V, maxiter, False


def calibrate(vobs, pi, pj, alpha, types, L, solver="lincal", tol=1e-10, maxiter=None, sparse=False):
    """Start point, solver and output convention for one channel.  sparse
    (lincal only): sparse linear algebra for the start point and the
    Gauss-Newton steps -- same equations, for large arrays.  L: the grid side,
    or the [N, 2] lattice coordinates of the antennas (see _pos)."""
    g0, V0 = initial_solution(vobs, pi, pj, alpha, types, L, sparse=sparse)
    if solver == "lincal":
        g, V, it, ok = lincal(vobs, pi, pj, alpha, g0, V0, types, L, tol=tol,
                              maxiter=maxiter or 200, sparse=sparse)
    elif solver == "omnical":
        g, V, it, ok = omnical(vobs, pi, pj, alpha, g0, V0, tol=tol, maxiter=maxiter or 100000)
    else:
        raise ValueError(solver)
    g, V = project(g, V, types, L)
    return g, V, it, ok


# --------------------------------------------------------------------------- covariance
def logcal_matrices(L, types, pi, pj, alpha):
    """Amplitude and phase design matrices of Eq. logcal (real parts)."""
    N, nu, P = L * L, len(types), len(pi)
    A = np.zeros((P, N + nu))
    B = np.zeros((P, N + nu))
    r = np.arange(P)
    np.add.at(A, (r, pi), 1.0)
    np.add.at(A, (r, pj), 1.0)
    np.add.at(A, (r, N + alpha), 1.0)
    np.add.at(B, (r, pi), 1.0)
    np.add.at(B, (r, pj), -1.0)
    np.add.at(B, (r, N + alpha), 1.0)
    return A, B


def logcal_normal_matrices(N, types, pi, pj, alpha):
    """A^T A and B^T B of Eq. logcal for N antennas, summed pair by pair
    (the outer products of the rows e_i + e_j + e_alpha and e_i - e_j +
    e_alpha): the same integers as A.T @ A and B.T @ B without forming the
    P x (N + n_ubl) design matrices, for arrays with many pairs."""
    nu = len(types)
    pi, pj = np.asarray(pi, np.int64), np.asarray(pj, np.int64)
    ka = N + np.asarray(alpha, np.int64)
    AtA = np.zeros((N + nu, N + nu))
    BtB = np.zeros((N + nu, N + nu))
    idx = [pi, pj, ka]
    sa = [1.0, 1.0, 1.0]
    sb = [1.0, -1.0, 1.0]
    for u in range(3):
        for v in range(3):
            np.add.at(AtA, (idx[u], idx[v]), sa[u] * sa[v])
            np.add.at(BtB, (idx[u], idx[v]), sb[u] * sb[v])
    return AtA, BtB


def gain_variance_prediction(L, types, pi, pj, alpha, N=None):
    """diag[(A^T A)^+]_{N x N} of Eq. gaincov, amplitude + phase parts.

    The pseudo-inverse leaves out the degenerate directions, which the
    paper's comparison fixes against the true gains.  N: antennas when the
    pair indices are not those of an L x L grid (e.g. a hexagonal array in
    its occupied-point numbering); default L * L.
    """
    N = L * L if N is None else N
    AtA, BtB = logcal_normal_matrices(N, types, pi, pj, alpha)
    # the exact degeneracies (Sec. 5.2) are singular values at rounding level;
    # a relative cut-off of 1e-9 leaves them out (the smallest physical
    # singular values of these normal matrices are ~1e-4 of the largest)
    ca = np.linalg.pinv(AtA, rcond=1e-9, hermitian=True)
    cb = np.linalg.pinv(BtB, rcond=1e-9, hermitian=True)
    return np.diag(ca)[:N], np.diag(cb)[:N]
