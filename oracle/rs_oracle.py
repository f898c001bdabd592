"""FP64 CPU oracle of the range-separated (RS) tensor method for the N-particle
Newton potential sum (Benner, Khoromskaia, Khoromskij, arXiv:1606.09218).

TEST INFRASTRUCTURE ONLY (see the package docstring).  Plain numpy/scipy, float64,
no blocking or fusion.  Each function names the passage of the paper it follows;
where the paper is silent or garbled the reading taken is stated in the docstring.

Notation follows the paper: b (half-width of the box), n (grid points per axis), h
(mesh size), t_k / a_k (sinc nodes / weights), p_k (1-D canonical factors of the
reference tensor P_R), R = R_l + R_s (long / short split), x_nu / z_nu (centres and
charges), U^(l) (side matrices), xi (canonical weights), Z0^(l) (Tucker bases),
beta (Tucker core), gamma (window half-width in grid steps).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf, erfc

SQRT_PI = math.sqrt(math.pi)


# ----------------------------------------------------------------------------
# Grid and quadrature  (Sec. 2.2)
# ----------------------------------------------------------------------------
def grid(b: float, n: int):
    """Vertex grid on [-b, b]: x_i = -b + i*h, i = 0..n-1, h = 2b/(n-1).

    Sec. 2.2 uses h = 2b/n with n even and the origin at the grid centre; with the
    odd sizes n = 2^k + 1 used here the centred vertex grid keeps the origin on a
    grid point (index (n-1)/2).  Reading: vertex grid with h = 2b/(n-1)."""
    h = 2.0 * b / (n - 1)
    return h, -b + h * np.arange(n, dtype=np.float64)


def sinc_quadrature(R: int, h_q: float, u0: float):
    """Nodes and weights of the sinc quadrature of the Laplace-Gauss transform
    1/z = (2/sqrt(pi)) * int_0^inf exp(-z^2 t^2) dt   (Sec. 2.2, Eqs. (2.6)-(2.8)).

    Eq. (2.7) prints t_k = k*h_M, a_k = a(t_k)*h_M, which taken literally puts a node
    at t = 0 whose constant term spoils 1/z away from the origin.  Reading: the
    exponential-sinc rule of the same transform after the substitution t = e^u,
    1/z = (2/sqrt(pi)) int_R exp(-z^2 e^{2u}) e^u du, sampled at u_k = u0 + k*h_q,
    k = 0..R-1, so t_k = exp(u_k) and a_k = (2/sqrt(pi)) * h_q * t_k (> 0).  Nodes are
    returned in increasing order of t_k."""
    k = np.arange(R, dtype=np.float64)
    t = np.exp(u0 + k * h_q)
    a = (2.0 / SQRT_PI) * h_q * t
    return t, a


def kernel_sum(t, a, rho):
    """sum_k a_k exp(-t_k^2 rho^2): the separable Gaussian-sum approximation of 1/rho
    (Sec. 2.2, Eq. (2.8)) evaluated at radii ``rho``."""
    rho = np.asarray(rho, dtype=np.float64)
    return (a[None, :] * np.exp(-(t[None, :] * rho.reshape(-1, 1)) ** 2)).sum(1).reshape(rho.shape)


def cell_average_gaussian(t: float, h: float, centre_offset):
    """(1/h) * int_{c-h/2}^{c+h/2} exp(-t^2 x^2) dx for cell centres c = ``centre_offset``.

    This is b_i(t_k)/h, the Galerkin projection of a 1-D Gaussian onto piecewise
    constant basis functions (Sec. 2.2, Eq. (2.5) and the definition of the vectors
    p_k^(l) before Eq. (2.10)), divided by the cell width.  Reading: cell averages
    (the projection divided by h) so that P_R approximates the cell average of 1/|x|
    rather than h^3 times it.  Closed form by the error function; the tail uses the
    complementary function erfc(x) = 1 - erf(x), with erf(b)-erf(a) = erfc(a)-erfc(b),
    to avoid the cancellation of two numbers close to one."""
    c = np.abs(np.asarray(centre_offset, dtype=np.float64))
    lo = t * (c - 0.5 * h)
    hi = t * (c + 0.5 * h)
    diff = np.where(lo > 0.5, erfc(lo) - erfc(hi), erf(hi) - erf(lo))
    return SQRT_PI / (2.0 * t * h) * diff


def reference_factors(t, a, h: float, n: int):
    """1-D factors of the reference canonical tensor on the doubled index range.

    Row k holds p_k[d] = a_k^{1/3} * (cell average of exp(-t_k^2 x^2) over the cell
    centred at d*h), d = -(n-1)..(n-1), stored at column d + n - 1.  P_R =
    sum_k p_k (x) p_k (x) p_k (Sec. 2.2, Eq. (2.10); the doubled grid of Sec. 3.2 that
    the shift-and-windowing transform of Eq. (3.4) reads from).  The three modes share
    the same vectors (Sec. 2.2, symmetry of the Newton kernel)."""
    d = np.arange(-(n - 1), n, dtype=np.float64) * h
    out = np.empty((len(t), 2 * n - 1))
    for k in range(len(t)):
        out[k] = a[k] ** (1.0 / 3.0) * cell_average_gaussian(t[k], h, d)
    return out


def split(R: int, R_s: int):
    """Index sets of the long- and short-range terms (Sec. 2.3, Eqs. (2.11)-(2.12)).

    Eq. (2.11) lists R_l + 1 long nodes and the text uses R_l + R_s = R.  Reading:
    R_l = R - R_s, the long part takes the R_l smallest t_k (k = 0..R_l-1) and the
    short part the R_s largest."""
    R_l = R - R_s
    return np.arange(R_l), np.arange(R_l, R)


def reference_value_at_origin(pk, kset, n: int):
    """P_R restricted to ``kset`` at the origin cell: sum_{k in kset} p_k[0]^3.
    Enters the self-interaction term of Eqs. (4.6)-(4.7) (Lemma 4.1)."""
    c = n - 1
    return float(np.sum(pk[kset, c] ** 3))


def window_halfwidth(pk, kshort, n: int, delta: float) -> int:
    """Half-width gamma (grid steps) of the cube that holds each short-range term.

    The short-range Gaussians are cut off where they fall below a threshold delta
    (Sec. 2.3, criterion (A), Eq. (2.13)); the windows are the gamma-vicinities of the
    cumulated canonical tensor (Def. 3.4, Def. 3.6).  Criterion (A) applied literally
    to all nodes would also pick the smallest t_k, so it is applied to the short set
    only.  Reading: gamma = min{g >= 0 : sum_{k short} p_k[g+1] * p_k[0]^2 <= delta},
    the largest value any truncated point (one coordinate offset > g, the others at
    the centre) could have carried, capped at n-1."""
    c = n - 1
    for g in range(0, n):
        if g + 1 > n - 1:
            return n - 1
        v = float(np.sum(pk[kshort, c + g + 1] * pk[kshort, c] ** 2))
        if v <= delta:
            return g
    return n - 1


def snap_to_grid(xyz, b: float, h: float, n: int):
    """Grid multi-index j^(nu) of each centre: the particle is moved to its nearest
    grid point (Sec. 3.2 assumes x_nu = h*j^(nu) on the grid).  Ties are rounded away
    from zero.  Raises if a centre lies outside [-b, b]^3."""
    xyz = np.asarray(xyz, dtype=np.float64)
    if np.any(np.abs(xyz) > b * (1 + 1e-12)):
        raise ValueError("particle outside the box")
    s = (xyz + b) / h
    j = np.floor(s + 0.5).astype(np.int64)
    return np.clip(j, 0, n - 1)


# ----------------------------------------------------------------------------
# Full-rank canonical sums (no range split, no truncation)  (Sec. 3.2, Eq. (3.4))
# ----------------------------------------------------------------------------
def canonical_sum_grid(j, z, pk, kset, n: int):
    """P = sum_nu z_nu W_nu(sum_{k in kset} p_k (x) p_k (x) p_k) on the whole n^3 grid,
    where W_nu shifts the reference tensor to the grid index j^(nu) (Sec. 3.2,
    Eqs. (3.4)-(3.5)).  kset = all R terms gives P_0, the long set gives P_l, the short
    set the untruncated P_s.  Computed as a plain sum of N*|kset| rank-one tensors,
    one matrix product per first index."""
    c = n - 1
    i = np.arange(n)
    cols = []
    for l in range(3):
        idx = i[:, None] - j[None, :, l] + c                  # (n, N)
        U = pk[kset][:, idx]                                  # (|kset|, n, N)
        cols.append(U.transpose(1, 2, 0).reshape(n, -1))      # (n, N*|kset|)
    w = np.repeat(np.asarray(z, dtype=np.float64), len(kset))
    P = np.empty((n, n, n))
    A = cols[1] * w[None, :]
    for i1 in range(n):
        P[i1] = (A * cols[0][i1][None, :]) @ cols[2].T
    return P


def canonical_sum_points(j, z, pk, kset, idx_pts, chunk: int = 256):
    """The same sum as ``canonical_sum_grid`` evaluated at the grid multi-indices
    ``idx_pts`` (M, 3) only (entry-wise definition of Eq. (3.4))."""
    n = (pk.shape[1] + 1) // 2
    c = n - 1
    idx_pts = np.asarray(idx_pts, dtype=np.int64)
    z = np.asarray(z, dtype=np.float64)
    out = np.empty(len(idx_pts))
    sub = pk[kset]
    for s in range(0, len(idx_pts), chunk):
        p = idx_pts[s:s + chunk]
        d = p[:, None, :] - j[None, :, :] + c                 # (m, N, 3)
        f = sub[:, d[..., 0]] * sub[:, d[..., 1]] * sub[:, d[..., 2]]   # (|k|, m, N)
        out[s:s + chunk] = np.einsum("kmn,n->m", f, z)
    return out


def direct_sum_points(xyz_src, z, pts):
    """P(x) = sum_nu z_nu / |x - x_nu|  (Sec. 1, Eq. (1.1); Sec. 3.1, Eq. (3.1)) at the
    points ``pts`` (M, 3).  Terms with |x - x_nu| = 0 are skipped."""
    pts = np.asarray(pts, dtype=np.float64)
    out = np.empty(len(pts))
    for s in range(0, len(pts), 512):
        d = pts[s:s + 512, None, :] - xyz_src[None, :, :]
        r = np.sqrt(np.einsum("mnk,mnk->mn", d, d))
        with np.errstate(divide="ignore"):
            inv = np.where(r > 0, 1.0 / np.where(r > 0, r, 1.0), 0.0)
        out[s:s + 512] = inv @ z
    return out


# ----------------------------------------------------------------------------
# Long-range side matrices and RHOSVD  (Sec. 3.2, Eq. (3.5); Sec. 6)
# ----------------------------------------------------------------------------
def side_matrices(j, z, pk, klong, n: int):
    """Side matrices U^(l) (n x N*R_l) and weights xi of the long-range canonical sum
    P_l = xi x_1 U^(1) x_2 U^(2) x_3 U^(3)  (Eq. (2.4) form of Eq. (3.5)).

    Column (nu, k) of U^(l) is w_nu * p_k[i - j_l^(nu)] with w_nu = |z_nu|^{1/3}; the sign
    of z_nu goes into xi.  The paper normalises the columns and keeps all weights in xi
    (Eq. (2.1)) without saying how xi enters the truncation.  Reading: the charge
    magnitude is spread evenly over the three modes."""
    c = n - 1
    i = np.arange(n)
    z = np.asarray(z, dtype=np.float64)
    w = np.abs(z) ** (1.0 / 3.0)
    Us = []
    for l in range(3):
        idx = i[:, None] - j[None, :, l] + c
        U = pk[klong][:, idx] * w[None, None, :]             # (R_l, n, N)
        Us.append(np.ascontiguousarray(U.transpose(1, 2, 0).reshape(n, -1)))
    xi = np.repeat(np.sign(z), len(klong))
    return Us, xi


def rhosvd_rank(sigma, eps: float, cap: int = 0) -> int:
    """Smallest r with sum_{k>r} sigma_k^2 <= (eps^2/3) * sum_k sigma_k^2, capped by ``cap``
    (> 0) and at least 1.  Sec. 6 (step (I) discards singular vectors "up to a given rank
    threshold" and mentions an eps-truncation criterion); the split of the budget into
    eps^2/3 per mode follows the sum over the three modes in the error bound of
    Lemma 3.12."""
    e2 = np.asarray(sigma, dtype=np.float64) ** 2
    total = e2.sum()
    tail = np.concatenate([np.cumsum(e2[::-1])[::-1], [0.0]])   # tail[r] = sum_{k>=r}
    thr = (eps * eps / 3.0) * total
    r = int(np.argmax(tail <= thr))
    r = max(r, 1)
    if cap and cap > 0:
        r = min(r, int(cap))
    return r


def rhosvd(Us, xi, eps: float, cap: int = 0, ranks=None):
    """Canonical-to-Tucker transform by the reduced HOSVD (Sec. 6, Eq. (6.1), Def. 6.1,
    Eqs. (6.2)-(6.3); no ALS sweeps, m_max = 0).

    (I)  SVD of each side matrix U^(l) = Z^(l) D_l V^(l)^T; keep the r_l dominant left
         singular vectors Z0^(l).
    (II) project, U~^(l) = Z0^(l)^T U^(l), and form the core
         beta = xi x_1 U~^(1) x_2 U~^(2) x_3 U~^(3).
    Returns (Z0 list, beta, ranks, singular values list)."""
    Z0s, sig, rk = [], [], []
    for l in range(3):
        Zl, s, _ = np.linalg.svd(Us[l], full_matrices=False)
        r = rhosvd_rank(s, eps, cap) if ranks is None else int(ranks[l])
        Z0s.append(Zl[:, :r])
        sig.append(s)
        rk.append(r)
    Y = [Z0s[l].T @ Us[l] for l in range(3)]
    beta = np.einsum("aK,bK,cK,K->abc", Y[0], Y[1], Y[2], xi, optimize=True)
    return Z0s, beta, rk, sig


def als_mode_matrix(Us, xi, Vs, l: int):
    """Partially projected image of the canonical tensor for mode l (Sec. 6, step (IV)):
    sum_K xi_K u_K^(l) (x) (V^(l')^T u_K^(l')) (x) (V^(l'')^T u_K^(l'')), with l' < l'' the two
    other modes, reshaped to the n x (r_l' r_l'') matrix M_{U_l} (column index b * r_l'' + c)."""
    o1, o2 = [m for m in range(3) if m != l]
    Y1 = Vs[o1].T @ Us[o1]                       # r_l' x K
    Y2 = Vs[o2].T @ Us[o2]                       # r_l'' x K
    M = np.einsum("iK,bK,cK,K->ibc", Us[l], Y1, Y2, xi, optimize=True)
    return M.reshape(Us[l].shape[0], -1)


def c2t_als(Us, xi, Z0s, eps: float, cap: int = 0, sweeps: int = 1, ranks=None):
    """ALS refinement of the canonical-to-Tucker transform (Sec. 6, steps (III)-(V)).

    Step (III) starts from the RHOSVD bases ``Z0s``.  Each sweep of step (IV) runs the modes in
    the order l = 1, 2, 3.  It forms M_{U_l} (``als_mode_matrix``) from the current bases of the
    other two modes and takes its SVD.  The r_l dominant left singular vectors become the new
    basis of mode l, so a later mode already sees the updated earlier ones.  r_l is the eps-rank of
    the singular values of M_{U_l} (the rule of ``rhosvd_rank``: the eps-truncation variant that
    the text allows), or ``ranks[l]`` when ranks are given.  Step (V) projects onto the final bases
    and forms the core.  Returns (bases, beta, ranks)."""
    Vs = [np.asarray(Z, dtype=np.float64) for Z in Z0s]
    rk = [V.shape[1] for V in Vs]
    for _ in range(int(sweeps)):
        for l in range(3):
            M = als_mode_matrix(Us, xi, Vs, l)
            Zl, s, _ = np.linalg.svd(M, full_matrices=False)
            r = rhosvd_rank(s, eps, cap) if ranks is None else int(ranks[l])
            Vs[l] = Zl[:, :r]
            rk[l] = r
    Y = [Vs[l].T @ Us[l] for l in range(3)]
    beta = np.einsum("aK,bK,cK,K->abc", Y[0], Y[1], Y[2], xi, optimize=True)
    return Vs, beta, rk


def tucker_full(beta, Vs):
    """beta x_1 V^(1) x_2 V^(2) x_3 V^(3) on the full grid (Eq. (2.3))."""
    return np.einsum("abc,ia,jb,kc->ijk", beta, Vs[0], Vs[1], Vs[2], optimize=True)


def tucker_points(beta, Vs, idx_pts):
    """Entries of the Tucker tensor at grid multi-indices (long-range term of Lemma 3.10)."""
    idx_pts = np.asarray(idx_pts, dtype=np.int64)
    A = Vs[0][idx_pts[:, 0]]
    B = Vs[1][idx_pts[:, 1]]
    C = Vs[2][idx_pts[:, 2]]
    return np.einsum("abc,ma,mb,mc->m", beta, A, B, C, optimize=True)


def canonical_norm2(Us, xi):
    """||P||_F^2 of a canonical tensor xi x_l U^(l):  xi^T (G1 * G2 * G3) xi with the
    column Gram matrices G_l = U^(l)^T U^(l)  (entry-wise product)."""
    G = (Us[0].T @ Us[0]) * (Us[1].T @ Us[1]) * (Us[2].T @ Us[2])
    return float(xi @ G @ xi)


# ----------------------------------------------------------------------------
# Short-range part: cumulated canonical tensor of windows  (Sec. 3.3)
# ----------------------------------------------------------------------------
def windows_full(j, z, pk, kshort, gamma: int, n: int):
    """Uniform cumulated canonical tensor sum_nu z_nu U_nu (Def. 3.4, Def. 3.6, Eq. (3.8)):
    U_nu is the short-range reference tensor sum_{k short} p_k (x) p_k (x) p_k shifted to
    j^(nu) and kept only on the cube |i_l - j_l^(nu)| <= gamma (clipped to the grid).
    Windows may overlap (the "soft" strategy of Example 3.5); overlaps add."""
    c = n - 1
    P = np.zeros((n, n, n))
    for nu in range(len(z)):
        if z[nu] == 0:
            continue
        lo = np.maximum(j[nu] - gamma, 0)
        hi = np.minimum(j[nu] + gamma, n - 1)
        f = []
        for l in range(3):
            d = np.arange(lo[l], hi[l] + 1) - j[nu, l] + c
            f.append(pk[kshort][:, d])                         # (R_s, len)
        block = np.einsum("ka,kb,kc->abc", f[0], f[1], f[2])
        P[lo[0]:hi[0] + 1, lo[1]:hi[1] + 1, lo[2]:hi[2] + 1] += z[nu] * block
    return P


def windows_points(j, z, pk, kshort, gamma: int, idx_pts):
    """Short-range entries sum_{nu in L(i)} c_nu U_nu(i) at grid multi-indices, where L(i)
    lists the windows that contain i (Lemma 3.10, second term)."""
    n = (pk.shape[1] + 1) // 2
    c = n - 1
    idx_pts = np.asarray(idx_pts, dtype=np.int64)
    out = np.zeros(len(idx_pts))
    sub = pk[kshort]
    for s in range(0, len(idx_pts), 256):
        p = idx_pts[s:s + 256]
        d = p[:, None, :] - j[None, :, :]                      # (m, N, 3)
        inside = np.all(np.abs(d) <= gamma, axis=2) & (np.asarray(z)[None, :] != 0)
        dd = d + c
        f = sub[:, dd[..., 0]] * sub[:, dd[..., 1]] * sub[:, dd[..., 2]]
        out[s:s + 256] = np.einsum("kmn,mn,n->m", f, inside.astype(np.float64), z)
    return out


def tucker_to_canonical(beta, Vs, eps: float):
    """Canonical form of the Tucker tensor beta x_1 V^(1) x_2 V^(2) x_3 V^(3), the long-range
    part of an RS-canonical tensor (Def. 3.7).  Sec. 3 reports RS-canonical ranks after a
    Tucker-to-canonical step at a given accuracy but does not state the algorithm.  Reading:
    the singular value decomposition of every mode-1 slice of the core,
    beta[a, :, :] = sum_m s_{a,m} x_{a,m} y_{a,m}^T; all (a, m) terms are ordered by s^2 and
    the smallest are discarded while their squared sum stays <= eps^2 ||beta||_F^2; every kept
    term is the rank-1 tensor s (V^(1) e_a) x (V^(2) x_{a,m}) x (V^(3) y_{a,m}).  With
    orthonormal V^(l) the Frobenius error is exactly sqrt(discarded) <= eps ||beta||_F.
    Returns (xi (R*), [U1, U2, U3] (n x R*), kept (a, m) pairs, discarded squared sum)."""
    beta = np.asarray(beta, dtype=np.float64)
    r1 = beta.shape[0]
    svd = [np.linalg.svd(beta[a], full_matrices=False) for a in range(r1)]
    terms = [(a, m, float(svd[a][1][m])) for a in range(r1) for m in range(len(svd[a][1]))]
    s2 = np.array([t[2] ** 2 for t in terms])
    budget = eps * eps * float(np.sum(beta * beta))
    order = np.argsort(s2, kind="stable")
    csum = np.cumsum(s2[order])
    ndisc = int(np.searchsorted(csum, budget, side="right"))
    drop = np.zeros(len(terms), dtype=bool)
    drop[order[:ndisc]] = True
    kept = [(a, m) for (a, m, _), d in zip(terms, drop) if not d]
    xi = np.array([svd[a][1][m] for a, m in kept])
    U1 = np.stack([Vs[0][:, a] for a, m in kept], axis=1) if kept else np.zeros((Vs[0].shape[0], 0))
    U2 = np.stack([Vs[1] @ svd[a][0][:, m] for a, m in kept], axis=1) if kept else np.zeros((Vs[1].shape[0], 0))
    U3 = np.stack([Vs[2] @ svd[a][2][m, :] for a, m in kept], axis=1) if kept else np.zeros((Vs[2].shape[0], 0))
    return xi, [U1, U2, U3], kept, float(csum[ndisc - 1]) if ndisc else 0.0


def canonical_full(xi, Us):
    """sum_k xi_k u_k^(1) x u_k^(2) x u_k^(3) on the full grid (first term of Eq. (3.10))."""
    return np.einsum("k,ik,jk,lk->ijl", xi, Us[0], Us[1], Us[2], optimize=True)


def canonical_points(xi, Us, idx_pts):
    """Entries of the canonical tensor at grid multi-indices: the Hadamard product of the rows
    of the three side matrices times xi (Lemma 3.8, first term)."""
    idx_pts = np.asarray(idx_pts, dtype=np.int64)
    return (Us[0][idx_pts[:, 0]] * Us[1][idx_pts[:, 1]] * Us[2][idx_pts[:, 2]]) @ xi


# ----------------------------------------------------------------------------
# Energy and forces  (Sec. 4.2, Sec. 4.3)
# ----------------------------------------------------------------------------
def energy_direct(xyz, z):
    """E_N = 1/2 sum_j z_j sum_{k != j} z_k / |x_j - x_k|   (Sec. 4.2, Eq. (4.4))."""
    xyz = np.asarray(xyz, dtype=np.float64)
    z = np.asarray(z, dtype=np.float64)
    E = 0.0
    for s in range(0, len(z), 1024):
        d = xyz[s:s + 1024, None, :] - xyz[None, :, :]
        r = np.sqrt(np.einsum("mnk,mnk->mn", d, d))
        rows = np.arange(s, min(s + 1024, len(z)))
        r[np.arange(len(rows)), rows] = np.inf
        E += float(z[rows] @ (1.0 / r) @ z)
    return 0.5 * E


def energy_scale(xyz, z):
    """sum_{j<k} |z_j z_k| / |x_j - x_k|: the size against which energy errors are
    measured (near-neutral systems make E_N itself small)."""
    return energy_direct(xyz, np.abs(z))


def energy_from_potential(p_at_particles, z, self_value):
    """E = 1/2 sum_j z_j (P(x_j) - z_j * P_ref(0))  (Sec. 4.2, Eq. (4.7) with P = P_0 and
    P_ref = P_R; Eq. (4.6), Lemma 4.1, with P = P_l and P_ref = P_{R_l})."""
    z = np.asarray(z, dtype=np.float64)
    return 0.5 * float(np.sum(z * (np.asarray(p_at_particles) - z * self_value)))


def forces_direct(xyz, z):
    """F_j = -dE_N/dx_j = z_j sum_{k != j} z_k (x_j - x_k) / |x_j - x_k|^3.

    Sec. 4.3 prints a factor 1/2 in front of this sum; differentiating Eq. (4.4), in
    which every pair appears twice, gives none.  Reading: no factor 1/2 (pinned by a
    finite-difference test of ``energy_direct``)."""
    xyz = np.asarray(xyz, dtype=np.float64)
    z = np.asarray(z, dtype=np.float64)
    F = np.zeros_like(xyz)
    for s in range(0, len(z), 1024):
        d = xyz[s:s + 1024, None, :] - xyz[None, :, :]
        r2 = np.einsum("mnk,mnk->mn", d, d)
        rows = np.arange(s, min(s + 1024, len(z)))
        r2[np.arange(len(rows)), rows] = np.inf
        w = z[None, :] / (r2 * np.sqrt(r2))
        F[rows] = z[rows, None] * np.einsum("mn,mnk->mk", w, d)
    return F


def gaussian_pair_energy(xyz, z, t, a, kset):
    """1/2 sum_{j != nu} z_j z_nu K(x_j - x_nu) with K(r) = sum_{k in kset} a_k exp(-t_k^2 |r|^2):
    the pair-sum form of Eq. (4.6) for collocated (continuous) Gaussians, where the
    self term z_j^2 K(0) cancels exactly (Lemma 4.1)."""
    xyz = np.asarray(xyz, dtype=np.float64)
    z = np.asarray(z, dtype=np.float64)
    E = 0.0
    for s in range(0, len(z), 512):
        d = xyz[s:s + 512, None, :] - xyz[None, :, :]
        r2 = np.einsum("mnk,mnk->mn", d, d)
        K = np.zeros_like(r2)
        for k in kset:
            K += a[k] * np.exp(-t[k] ** 2 * r2)
        rows = np.arange(s, min(s + 512, len(z)))
        K[np.arange(len(rows)), rows] = 0.0
        E += float(z[rows] @ K @ z)
    return 0.5 * E


def gaussian_pair_forces(xyz, z, t, a, kset):
    """-d/dx_j of ``gaussian_pair_energy``:
    F_j = z_j sum_{nu != j} z_nu sum_k 2 a_k t_k^2 (x_j - x_nu) exp(-t_k^2 |x_j - x_nu|^2),
    i.e. F_j = -z_j grad P_kset(x_j) with the self term removed (Sec. 4.3)."""
    xyz = np.asarray(xyz, dtype=np.float64)
    z = np.asarray(z, dtype=np.float64)
    F = np.zeros_like(xyz)
    for s in range(0, len(z), 512):
        d = xyz[s:s + 512, None, :] - xyz[None, :, :]
        r2 = np.einsum("mnk,mnk->mn", d, d)
        W = np.zeros_like(r2)
        for k in kset:
            W += 2.0 * a[k] * t[k] ** 2 * np.exp(-t[k] ** 2 * r2)
        rows = np.arange(s, min(s + 512, len(z)))
        W[np.arange(len(rows)), rows] = 0.0
        F[rows] = z[rows, None] * np.einsum("mn,n,mnk->mk", W, z, d)
    return F


# ----------------------------------------------------------------------------
# Galerkin kernel off the grid and the adjoint forces  (Sec. 4.3)
# ----------------------------------------------------------------------------
def cell_average_gaussian_derivative(t: float, h: float, centre_offset):
    """d/dc of ``cell_average_gaussian``: the cell average (1/h) int_{c-h/2}^{c+h/2} exp(-t^2 x^2) dx
    differentiated in its centre c is, by the fundamental theorem of calculus,
    (exp(-t^2 (c + h/2)^2) - exp(-t^2 (c - h/2)^2)) / h."""
    c = np.asarray(centre_offset, dtype=np.float64)
    return (np.exp(-(t * (c + 0.5 * h)) ** 2) - np.exp(-(t * (c - 0.5 * h)) ** 2)) / h


def galerkin_factors_at(t, a, h: float, y, derivative: bool = False):
    """p_k(y) = a_k^{1/3} * (cell average of exp(-t_k^2 x^2) over the cell centred at y) for any
    offsets y (leading axis over k), or its derivative in y.  On grid offsets y = d*h these are
    the entries of ``reference_factors`` (Eq. (2.10)); off the grid they extend the grid tensor
    P_R continuously in the centre position (reading used for the adjoint forces of Sec. 4.3)."""
    y = np.asarray(y, dtype=np.float64)
    f = cell_average_gaussian_derivative if derivative else cell_average_gaussian
    out = np.empty((len(t),) + y.shape)
    for k in range(len(t)):
        out[k] = a[k] ** (1.0 / 3.0) * f(t[k], h, y)
    return out


def galerkin_pair_energy(xyz, z, t, a, kset, h: float):
    """1/2 sum_{j != nu} z_j z_nu K_h(x_j - x_nu) with the Galerkin RS kernel
    K_h(r) = sum_{k in kset} p_k(r_1) p_k(r_2) p_k(r_3)  (the continuous form of P_R, Eq. (2.10),
    from ``galerkin_factors_at``); pair-sum form of Eq. (4.6), the self term cancels (Lemma 4.1)."""
    xyz = np.asarray(xyz, dtype=np.float64)
    z = np.asarray(z, dtype=np.float64)
    tk, ak = t[kset], a[kset]
    E = 0.0
    for s in range(0, len(z), 256):
        d = xyz[s:s + 256, None, :] - xyz[None, :, :]
        f = [galerkin_factors_at(tk, ak, h, d[:, :, l]) for l in range(3)]
        K = (f[0] * f[1] * f[2]).sum(0)
        rows = np.arange(s, min(s + 256, len(z)))
        K[np.arange(len(rows)), rows] = 0.0
        E += float(z[rows] @ K @ z)
    return 0.5 * E


def galerkin_pair_forces(xyz, z, t, a, kset, h: float):
    """-d/dx_j of ``galerkin_pair_energy``: F_j = -z_j sum_{nu != j} z_nu grad K_h(x_j - x_nu)
    (each pair appears twice in the energy; Sec. 4.3 with the spurious 1/2 of the printed force
    formula removed)."""
    xyz = np.asarray(xyz, dtype=np.float64)
    z = np.asarray(z, dtype=np.float64)
    tk, ak = t[kset], a[kset]
    F = np.zeros_like(xyz)
    for s in range(0, len(z), 256):
        d = xyz[s:s + 256, None, :] - xyz[None, :, :]
        f = [galerkin_factors_at(tk, ak, h, d[:, :, l]) for l in range(3)]
        g = [galerkin_factors_at(tk, ak, h, d[:, :, l], derivative=True) for l in range(3)]
        rows = np.arange(s, min(s + 256, len(z)))
        for l in range(3):
            prod = g[l] * f[(l + 1) % 3] * f[(l + 2) % 3]
            dK = prod.sum(0)
            dK[np.arange(len(rows)), rows] = 0.0
            F[rows, l] = -z[rows] * (dK @ z)
    return F


def rs_tucker_forces(j, z, pk, dpk, klong, kshort, gamma: int, Us, Z0s, beta, n: int):
    """Adjoint forces of the RS-Tucker energy at snapped centres (Sec. 4.3 applied to
    Def. 3.9 / Lemma 3.10):  F_j = -z_j [grad P_l^T(x_j) + sum_{nu != j, window} z_nu grad P_s,nu(x_j)].

    The long-range part P_l^T = beta x_l V^(l) is differentiated through the continuous form of
    its Tucker vectors: with U^(l) = Z D W^T (SVD), Z0^(l) = U^(l) W D^{-1}, so each basis vector
    is a combination of the side-matrix columns, v_a(y) = sum_K u_K(y) (U^T Z0)[K, a] / sigma_a^2,
    and v_a'(y) uses the derivative factors ``dpk`` (rows of ``galerkin_factors_at`` with
    derivative=True on the doubled grid).  (Projecting the derivative factor vectors onto the
    Tucker subspaces instead does not converge with eps: the subspaces are built for the
    factors, not for their derivatives.)  The short-range part is the window sum of Def. 3.4
    differentiated term by term.  ``Us`` are the side matrices of ``side_matrices``."""
    c = n - 1
    z = np.asarray(z, dtype=np.float64)
    w = np.abs(z) ** (1.0 / 3.0)
    N = len(z)
    V, Vd = [], []
    for l in range(3):
        Y = Us[l].T @ Z0s[l]                                   # (N*R_l, r): (U^T Z0)
        s2 = np.einsum("Ka,Ka->a", Y, Y)                       # ||U^T z_a||^2 = sigma_a^2
        i = j[:, l]
        # derivative columns u_K'(x_i) for K = (nu, k): w_nu * dp_k[i - j_nu]
        idx = i[:, None] - j[None, :, l] + c                   # (N, N)
        dU = dpk[klong][:, idx] * w[None, None, :]             # (R_l, N, N): [k][point][nu]
        dU = dU.transpose(1, 2, 0).reshape(N, -1)              # (point, (nu, k))
        Vd.append(dU @ Y / s2[None, :])
        V.append(Z0s[l][i])
    F = np.zeros((N, 3))
    grads = [np.einsum("abc,ma,mb,mc->m", beta, Vd[0], V[1], V[2], optimize=True),
             np.einsum("abc,ma,mb,mc->m", beta, V[0], Vd[1], V[2], optimize=True),
             np.einsum("abc,ma,mb,mc->m", beta, V[0], V[1], Vd[2], optimize=True)]
    for l in range(3):
        F[:, l] = -z * grads[l]
    # short-range windows of the other particles
    for m in range(N):
        dj = j[m][None, :] - j                                 # (N, 3)
        near = np.all(np.abs(dj) <= gamma, axis=1)
        near[m] = False
        if not near.any():
            continue
        d = dj[near] + c
        f = [pk[kshort][:, d[:, l]] for l in range(3)]
        g = [dpk[kshort][:, d[:, l]] for l in range(3)]
        for l in range(3):
            dP = (g[l] * f[(l + 1) % 3] * f[(l + 2) % 3]).sum(0)
            F[m, l] -= z[m] * float(dP @ z[near])
    return F


def rs_direct_long_forces(j, z, pk, dpk, klong, kshort, gamma: int, n: int):
    """Forces of the untruncated long-range canonical sum plus the windows at snapped centres:
    F_j = -z_j [grad P_l(x_j) + window terms], grad P_l(x_j) = sum_{nu != j} z_nu sum_{k long}
    grad (p_k (x) p_k (x) p_k)(x_j - x_nu) with the Galerkin factors and their derivatives on the
    grid offsets (F = -z grad P_l of Sec. 4.3, exact for P_l by symmetry)."""
    c = n - 1
    z = np.asarray(z, dtype=np.float64)
    N = len(z)
    F = np.zeros((N, 3))
    for m in range(N):
        d = j[m][None, :] - j + c                              # (N, 3)
        f = [pk[klong][:, d[:, l]] for l in range(3)]
        g = [dpk[klong][:, d[:, l]] for l in range(3)]
        zz = z.copy()
        zz[m] = 0.0
        for l in range(3):
            F[m, l] = -z[m] * float((g[l] * f[(l + 1) % 3] * f[(l + 2) % 3]).sum(0) @ zz)
        dj = j[m][None, :] - j
        near = np.all(np.abs(dj) <= gamma, axis=1)
        near[m] = False
        if near.any():
            ds = dj[near] + c
            fs = [pk[kshort][:, ds[:, l]] for l in range(3)]
            gs = [dpk[kshort][:, ds[:, l]] for l in range(3)]
            for l in range(3):
                F[m, l] -= z[m] * float((gs[l] * fs[(l + 1) % 3] * fs[(l + 2) % 3]).sum(0) @ z[near])
    return F


def reference_factor_derivatives(t, a, h: float, n: int):
    """Derivatives in the centre offset of the rows of ``reference_factors`` on the doubled grid
    (``galerkin_factors_at`` with derivative=True at y = d*h, d = -(n-1)..(n-1))."""
    d = np.arange(-(n - 1), n, dtype=np.float64) * h
    return galerkin_factors_at(t, a, h, d, derivative=True)


# ----------------------------------------------------------------------------
# Discrete gradient of the RS tensor and the forces from it  (Sec. 4.3, Eq. (4.9))
# ----------------------------------------------------------------------------
def fd_first_derivative_weights(offsets, h: float):
    """Weights w of the first-derivative difference formula on the given integer offsets,
    sum_s w_s f(x + s h) ~ f'(x), from the Taylor conditions: sum_s w_s s^q = [q == 1] / h for
    q = 0 .. len(offsets) - 1 (exact for polynomials of that degree).  Sec. 4.3 applies a
    one-dimensional difference operator (backward or central) to the canonical vectors; the
    order is a parameter here."""
    s = np.asarray(offsets, dtype=np.float64)
    m = len(s)
    A = np.vander(s, m, increasing=True).T             # A[q][i] = s_i^q
    rhs = np.zeros(m)
    rhs[1] = 1.0
    return np.linalg.solve(A, rhs) / h


def fd_matrix(n: int, h: float, order: int = 8):
    """The n x n matrix D_h of the first-derivative difference operator on the grid: row i uses
    the order + 1 consecutive grid points centred on i where they fit, else the window of that
    width nearest to i inside the grid (one-sided near the ends).  Reading: Sec. 4.3 names
    backward or central differences; centred formulas of order ``order`` are used in the
    interior, and the same width is kept at the ends of the grid."""
    width = order + 1
    D = np.zeros((n, n))
    for i in range(n):
        start = min(max(i - order // 2, 0), n - width)
        cols = np.arange(start, start + width)
        D[i, cols] = fd_first_derivative_weights(cols - i, h)
    return D


def canonical_fd_gradient_points(j, z, pk, kset, D, idx_pts):
    """Discrete gradient (D_h applied along each mode, Sec. 4.3, Eq. (4.9)) of the full-rank
    canonical sum sum_nu z_nu sum_{k in kset} p_k (x) p_k (x) p_k shifted to j^(nu), at the grid
    multi-indices idx_pts (M, 3): returns (M, 3).  Each term's mode-l factor vector is replaced by
    its difference D_h p_k(. - j_l^(nu)), written out per point and stencil entry."""
    n = D.shape[0]
    c = n - 1
    idx_pts = np.asarray(idx_pts, dtype=np.int64)
    z = np.asarray(z, dtype=np.float64)
    sub = pk[kset]
    out = np.zeros((len(idx_pts), 3))
    for m, p in enumerate(idx_pts):
        f = [sub[:, p[l] - j[:, l] + c] for l in range(3)]            # (|k|, N) factor values
        for l in range(3):
            cols = np.nonzero(D[p[l]])[0]
            df = np.zeros_like(f[l])
            for q in cols:
                df += D[p[l], q] * sub[:, q - j[:, l] + c]
            out[m, l] = float(((df * f[(l + 1) % 3] * f[(l + 2) % 3]).sum(0)) @ z)
    return out


def fd_self_gradient(j, pk, kset, D):
    """D_h of the particle's own term sum_k p_k (x) p_k (x) p_k at its own grid point, per mode
    (N, 3): zero for a centred formula (the term is even), the small value of a one-sided
    formula near the ends of the grid.  The forces leave the particle's own term out."""
    n = D.shape[0]
    c = n - 1
    sub = pk[kset]
    p0 = sub[:, c]
    out = np.zeros((len(j), 3))
    for m in range(len(j)):
        for l in range(3):
            i = j[m, l]
            cols = np.nonzero(D[i])[0]
            df = sum(D[i, q] * sub[:, q - i + c] for q in cols)
            out[m, l] = float((df * p0 * p0).sum())
    return out


def _window_forces(j, z, pk, dpk, kshort, gamma: int, n: int):
    """Short-range part of the forces: the windows of the other particles (Def. 3.4)
    differentiated term by term with the derivative factors, -z_m sum_{nu != m} z_nu grad U_nu."""
    c = n - 1
    z = np.asarray(z, dtype=np.float64)
    F = np.zeros((len(z), 3))
    for m in range(len(z)):
        dj = j[m][None, :] - j
        near = np.all(np.abs(dj) <= gamma, axis=1)
        near[m] = False
        if not near.any():
            continue
        d = dj[near] + c
        f = [pk[kshort][:, d[:, l]] for l in range(3)]
        g = [dpk[kshort][:, d[:, l]] for l in range(3)]
        for l in range(3):
            F[m, l] -= z[m] * float((g[l] * f[(l + 1) % 3] * f[(l + 2) % 3]).sum(0) @ z[near])
    return F


def canonical_fd_forces(j, z, pk, dpk, klong, kshort, gamma: int, D):
    """Forces from the discrete gradient of the untruncated long-range canonical sum (Sec. 4.3):
    F_m = -z_m [D_h P_l(x_m) - z_m D_h K_l(0)] - z_m sum_{nu != m, window} z_nu grad U_nu(x_m),
    the particle's own long-range term taken out, the windows differentiated term by term."""
    n = D.shape[0]
    z = np.asarray(z, dtype=np.float64)
    G = canonical_fd_gradient_points(j, z, pk, klong, D, j)
    G -= z[:, None] * fd_self_gradient(j, pk, klong, D)
    return -z[:, None] * G + _window_forces(j, z, pk, dpk, kshort, gamma, n)


def rs_tucker_fd_forces(j, z, pk, dpk, klong, kshort, gamma: int, Z0s, beta, D):
    """Forces from the discrete gradient of the RS-Tucker tensor (Sec. 4.3, Eq. (4.9) applied to
    the Tucker form of Def. 3.9): the mode-l derivative of P_l^T = beta x_1 V1 x_2 V2 x_3 V3 is
    beta with V_l replaced by D_h V_l, evaluated at the particle's grid point,
    F_m = -z_m [(D_h P_l^T)(x_m) - z_m D_h K_l(0)] + window terms as in canonical_fd_forces."""
    n = D.shape[0]
    z = np.asarray(z, dtype=np.float64)
    dV = [D @ V for V in Z0s]
    V = [Z0s[l][j[:, l]] for l in range(3)]
    Vd = [dV[l][j[:, l]] for l in range(3)]
    G = np.stack([np.einsum("abc,ma,mb,mc->m", beta, Vd[0], V[1], V[2], optimize=True),
                  np.einsum("abc,ma,mb,mc->m", beta, V[0], Vd[1], V[2], optimize=True),
                  np.einsum("abc,ma,mb,mc->m", beta, V[0], V[1], Vd[2], optimize=True)], axis=1)
    G -= z[:, None] * fd_self_gradient(j, pk, klong, D)
    return -z[:, None] * G + _window_forces(j, z, pk, dpk, kshort, gamma, n)


# ----------------------------------------------------------------------------
# RS interaction matrix and its matrix-vector product  (Sec. 4.1 problem (B), Sec. 4.2)
# ----------------------------------------------------------------------------
def toeplitz_factor(pk_row, n: int, cut: int = -1):
    """The n x n symmetric Toeplitz matrix T[i][i'] = p_k[i - i'] generated by one factor vector
    (Sec. 4.1, case (A): the univariate matrices A_k^(l) of the Kronecker product sum), with the
    entries beyond |i - i'| > cut set to zero when cut >= 0 (the window of a short-range term,
    Def. 3.4)."""
    c = n - 1
    i = np.arange(n)
    d = i[:, None] - i[None, :]
    T = pk_row[d + c].copy()
    if cut >= 0:
        T[np.abs(d) > cut] = 0.0
    return T


def rs_matrix_dense(pk, klong, kshort, gamma: int, n: int):
    """The RS interaction matrix of the n^3 grid points, A = A_l + A_s (Sec. 4.1, case (A)), as a
    dense n^3 x n^3 array (C order, i3 fastest): the long part is the R_l-term Kronecker product
    sum of Toeplitz factors, A_l = sum_{k long} T_k (x) T_k (x) T_k; the short part keeps the
    R_s short terms inside the window |i_l - i'_l| <= gamma of every mode (the cumulated
    canonical tensor of Defs. 3.4, 3.6), A_s = sum_{k short} T_k^gamma (x) T_k^gamma (x) T_k^gamma.
    For small n only (n^6 entries)."""
    N3 = n ** 3
    A = np.zeros((N3, N3))
    for k in klong:
        T = toeplitz_factor(pk[k], n)
        A += np.kron(np.kron(T, T), T)
    for k in kshort:
        T = toeplitz_factor(pk[k], n, gamma)
        A += np.kron(np.kron(T, T), T)
    return A


def rs_matvec_dense(pk, klong, kshort, gamma: int, n: int, X, offdiag: bool = False):
    """Y = A X with the dense RS interaction matrix (X an n^3 tensor); with ``offdiag`` the
    diagonal part diag(A) X is left out (the matrix A - diag A of Eq. (4.6))."""
    A = rs_matrix_dense(pk, klong, kshort, gamma, n)
    if offdiag:
        A = A - np.diag(np.diag(A))
    return (A @ np.asarray(X, dtype=np.float64).ravel()).reshape((n, n, n))


def charge_grid(j, z, n: int):
    """The charges as an n^3 tensor: z_nu at the grid point j^(nu) (added if several share it)."""
    C = np.zeros((n, n, n))
    np.add.at(C, (j[:, 0], j[:, 1], j[:, 2]), np.asarray(z, dtype=np.float64))
    return C


def energy_matvec(pk, klong, kshort, gamma: int, n: int, j, z):
    """E_N = 1/2 <(A - diag A) z, z> (Sec. 4.2, Eq. (4.6)) with the RS interaction matrix of the
    grid and z the charges embedded in the grid (distinct grid points)."""
    C = charge_grid(j, z, n)
    Y = rs_matvec_dense(pk, klong, kshort, gamma, n, C, offdiag=True)
    return 0.5 * float(np.sum(C * Y))


# ----------------------------------------------------------------------------
# Whole-problem driver used by the tests
# ----------------------------------------------------------------------------
class Problem:
    """All reference quantities of one snapped particle set under one parameter set.

    ``cfg`` keys: b, n, R, R_s, h_q, u0, eps, rank_cap, delta_rel."""

    def __init__(self, cfg: dict, xyz, z):
        self.cfg = cfg
        self.b = float(cfg["b"])
        self.n = int(cfg["n"])
        self.R = int(cfg["R"])
        self.R_s = int(cfg["R_s"])
        self.h, self.x = grid(self.b, self.n)
        self.t, self.a = sinc_quadrature(self.R, float(cfg["h_q"]), float(cfg["u0"]))
        self.pk = reference_factors(self.t, self.a, self.h, self.n)
        self.klong, self.kshort = split(self.R, self.R_s)
        self.kall = np.arange(self.R)
        self.PR0 = reference_value_at_origin(self.pk, self.kall, self.n)
        self.PRl0 = reference_value_at_origin(self.pk, self.klong, self.n)
        self.delta = float(cfg["delta_rel"]) * self.PR0
        self.gamma = window_halfwidth(self.pk, self.kshort, self.n, self.delta)
        self.xyz = np.asarray(xyz, dtype=np.float64)
        self.z = np.asarray(z, dtype=np.float64)
        self.j = snap_to_grid(self.xyz, self.b, self.h, self.n)
        self.xyz_snapped = self.x[self.j]

    # full-rank canonical sums
    def P0_grid(self):
        return canonical_sum_grid(self.j, self.z, self.pk, self.kall, self.n)

    def Pl_grid(self):
        return canonical_sum_grid(self.j, self.z, self.pk, self.klong, self.n)

    def Ps_grid(self):
        return canonical_sum_grid(self.j, self.z, self.pk, self.kshort, self.n)

    def P0_points(self, idx):
        return canonical_sum_points(self.j, self.z, self.pk, self.kall, idx)

    def Pl_points(self, idx):
        return canonical_sum_points(self.j, self.z, self.pk, self.klong, idx)

    # RS-Tucker
    def tucker(self, eps=None, cap=None, ranks=None):
        Us, xi = side_matrices(self.j, self.z, self.pk, self.klong, self.n)
        e = float(self.cfg["eps"]) if eps is None else eps
        c = int(self.cfg.get("rank_cap", 0)) if cap is None else cap
        Z0s, beta, rk, sig = rhosvd(Us, xi, e, c, ranks)
        return Z0s, beta, rk, sig, Us, xi

    def windows_grid(self):
        return windows_full(self.j, self.z, self.pk, self.kshort, self.gamma, self.n)

    def windows_points(self, idx):
        return windows_points(self.j, self.z, self.pk, self.kshort, self.gamma, idx)

    # energies
    def energy_direct_snapped(self):
        return energy_direct(self.xyz_snapped, self.z)

    def energy_P0(self):
        return energy_from_potential(self.P0_points(self.j), self.z, self.PR0)

    # forces (Sec. 4.3)
    def forces_galerkin(self, kset=None):
        """Adjoint forces of the untruncated Galerkin RS kernel at the snapped centres."""
        ks = self.kall if kset is None else kset
        return galerkin_pair_forces(self.xyz_snapped, self.z, self.t, self.a, ks, self.h)

    def forces_rs_tucker(self, ranks=None, eps=None):
        """Adjoint forces of the RS-Tucker tensor (long part at the given ranks + windows)."""
        Z0s, beta, rk, _, Us, _ = self.tucker(eps=eps, cap=0 if ranks is not None else None, ranks=ranks)
        dpk = reference_factor_derivatives(self.t, self.a, self.h, self.n)
        return rs_tucker_forces(self.j, self.z, self.pk, dpk, self.klong, self.kshort, self.gamma, Us,
                                Z0s, beta, self.n), rk

    def fd_matrix(self, order: int = 8):
        return fd_matrix(self.n, self.h, order)

    def forces_canonical_fd(self, order: int = 8):
        """Forces from the discrete gradient of the untruncated long-range sum (Sec. 4.3)."""
        dpk = reference_factor_derivatives(self.t, self.a, self.h, self.n)
        return canonical_fd_forces(self.j, self.z, self.pk, dpk, self.klong, self.kshort, self.gamma,
                                   self.fd_matrix(order))

    def forces_rs_tucker_fd(self, ranks=None, eps=None, order: int = 8, cap: int = 0):
        """Forces from the discrete gradient of the RS-Tucker tensor (Sec. 4.3, Def. 3.9), at the
        given ranks or at the eps ranks (capped by ``cap``, 0 = none)."""
        Z0s, beta, rk, _, _, _ = self.tucker(eps=eps, cap=cap, ranks=ranks)
        dpk = reference_factor_derivatives(self.t, self.a, self.h, self.n)
        return rs_tucker_fd_forces(self.j, self.z, self.pk, dpk, self.klong, self.kshort, self.gamma, Z0s, beta,
                                   self.fd_matrix(order)), rk

    def forces_direct_long(self):
        """Untruncated long-range forces plus windows at the snapped centres."""
        dpk = reference_factor_derivatives(self.t, self.a, self.h, self.n)
        return rs_direct_long_forces(self.j, self.z, self.pk, dpk, self.klong, self.kshort, self.gamma,
                                     self.n)
