"""FP64 CPU oracle for multi-scale range-image point-to-plane registration.

TEST INFRASTRUCTURE ONLY.  This module is the slow, plainly written reference
that the CUDA library is checked against.  Only the test-suite, the smoke check
and the benchmark's CPU-baseline leg may import it; the library never does,
and it shares no code, tables or helpers with the CUDA path.

Everything is float64 numpy, one array operation per step of the paper's
definitions, in the paper's order:

* unprojection Pi^-1, Eq. 1-2 (Section 3.1);
* projection Pi with the receiver-offset fixed point and the elevation argmin,
  Eq. 3-4 and the column recovery that reverts Eq. 2 (Section 3.2);
* the 2H-entry inverse elevation table of Section 3.2 (used only to pin the
  paper's +-1 claim; the projection itself uses the exact argmin of Eq. 4);
* projective data association, Eq. 5-6, the point-to-plane loss with a
  pseudo-Huber robust kernel and one Gauss-Newton step of Eq. 7
  (Section 4.1, kernel size from Section 6.1);
* normals as the cross product of neighbouring pixels' points (Section 4.1);
* the strided pyramid that keeps the sensor intrinsics (Section 4.1) and the
  coarse-to-fine schedule (Section 6.1).

Readings of points the paper leaves open (all listed in the design notes):
  - u = floor(u_c + 1/2) mod W, theta wrapped into [0, 2 pi) (Section 3.2
    footnote); elevation ties go to the lower row index.
  - The receiver offset is compensated at the *column* angle 2 pi u_c / W
    (Eq. 1 puts the receiver there), iterated to |du_c| < 1e-10 px or 50 steps.
  - A projected point is outside the image vertically when its elevation lies
    more than half an edge-row spacing beyond the first or last row of the
    level's table; horizontally the image wraps (360 degrees).
  - Normals: central differences a = P(u+1,v) - P(u-1,v) (u wraps),
    b = P(u,v+1) - P(u,v-1); n = a x b / |a x b|, flipped so n . P <= 0.
    Invalid on rows 0 and H-1, when any of the five ranges is invalid, when a
    neighbour's range differs from the centre's by more than rel_jump * r_c,
    or when |a x b| <= 1e-4 |a||b| (near-parallel differences).
  - Level l of the pyramid is the image strided by 2^l in both directions with
    the tables phi_lut[2^l v], theta_lut[2^l v], W_l = W / 2^l and the same r0;
    normals are strided, not recomputed.
  - Robust kernel rho(e) = d^2 (sqrt(1 + (e/d)^2) - 1) with IRLS weight
    w = 1 / sqrt(1 + (e/d)^2); d <= 0 means plain least squares (w = 1).
  - Left perturbation x <- Exp(xi) x, xi = (omega, tau), J = [x x n, n];
    T <- Exp(xi) T with xi = -(J^T W J)^-1 J^T W e.  A system with fewer than 6
    correspondences or a Cholesky pivot <= 1e-12 * trace leaves T unchanged.
  - A range is invalid when it is <= 0 or not finite.
"""
import numpy as np

TWO_PI = 2.0 * np.pi
NORMAL_SIN_EPS = 1e-4
CHOL_REL_EPS = 1e-12
NEAR_TIE_PX = 1e-3          # |u_c - (k + 1/2)| below this is a u near-tie (pixels)
NEAR_TIE_ROW = 1e-3         # elevation distance to a row boundary / row spacing


# ----------------------------------------------------------------------------
# Section 3.1: unprojection, Eq. 1-2

def level_tables(phi_lut, theta_lut, level):
    """Level-l tables of the strided pyramid: every 2^l-th row (Section 4.1)."""
    s = 1 << level
    return np.asarray(phi_lut, np.float64)[::s], np.asarray(theta_lut, np.float64)[::s]


def range_valid(r):
    r = np.asarray(r, np.float64)
    return np.isfinite(r) & (r > 0)


def unproject_pixels(u, v, r, phi_lut, theta_lut, r0, W):
    """Eq. 1-2 for arrays of integer columns u, rows v and ranges r -> (..., 3)."""
    u = np.asarray(u, np.float64)
    v = np.asarray(v, np.int64)
    r = np.asarray(r, np.float64)
    col = TWO_PI * u / W                      # receiver azimuth 2 pi u / W
    theta = col + theta_lut[v]                # Eq. 2: theta(u, v)
    phi = phi_lut[v]                          # Eq. 2: phi(v)
    x = r * np.cos(theta) * np.cos(phi) + r0 * np.cos(col)
    y = r * np.sin(theta) * np.cos(phi) + r0 * np.sin(col)
    z = r * np.sin(phi)
    return np.stack([x, y, z], axis=-1)


def unproject(range_img, phi_lut, theta_lut, r0):
    """Whole-image unprojection: points (H, W, 3) and validity mask (H, W).
    Invalid pixels get the point computed from r = 0 (masked out by callers)."""
    rimg = np.asarray(range_img, np.float64)
    H, W = rimg.shape
    valid = range_valid(rimg)
    r = np.where(valid, rimg, 0.0)
    vv, uu = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    return unproject_pixels(uu, vv, r, np.asarray(phi_lut, np.float64),
                            np.asarray(theta_lut, np.float64), r0, W), valid


# ----------------------------------------------------------------------------
# Section 3.2: projection, Eq. 3-4 and the inverse of Eq. 2

def row_argmin(phi, phi_lut):
    """Eq. 4: v = argmin_t |phi_lut[t] - phi| over all H rows (ties -> lower t)."""
    phi = np.asarray(phi, np.float64)
    d = np.abs(np.asarray(phi_lut, np.float64)[None, :] - phi.reshape(-1, 1))
    return np.argmin(d, axis=1).reshape(phi.shape)


def fov_limits(phi_lut):
    """Elevation interval that maps into the image: half an edge spacing beyond
    the highest and the lowest row of the table."""
    p = np.sort(np.asarray(phi_lut, np.float64))
    return p[0] - 0.5 * (p[1] - p[0]), p[-1] + 0.5 * (p[-1] - p[-2])


def row_margin(phi, phi_lut):
    """Distance of phi to the nearest decision boundary of the row choice (a
    midpoint between adjacent rows, or an edge of the field of view), in units
    of the local row spacing.  Used only to flag near-ties in parity tests."""
    p = np.sort(np.asarray(phi_lut, np.float64))
    mids = 0.5 * (p[1:] + p[:-1])
    gaps = p[1:] - p[:-1]
    lo, hi = fov_limits(phi_lut)
    bounds = np.concatenate([[lo], mids, [hi]])
    scale = np.concatenate([[gaps[0]], gaps, [gaps[-1]]])
    phi = np.asarray(phi, np.float64).reshape(-1, 1)
    return np.min(np.abs(phi - bounds[None, :]) / scale[None, :], axis=1)


def project(X, phi_lut, theta_lut, r0, W, max_iter=50, tol=1e-10, return_detail=False):
    """Pi(X) of Section 3.2 for points X (..., 3).

    r = |X - o|, phi = asin(z / r), theta = atan2 wrapped to [0, 2 pi);
    u_hat = W theta / 2 pi; the receiver offset o = r0 (cos, sin)(2 pi u_c / W)
    is compensated with the current column estimate and the estimate repeated
    until it converges; v by Eq. 4; u = u_hat - W theta_lut[v] / 2 pi, rounded
    half up and wrapped.

    Returns u (int), v (int), r, in_fov (bool) and, with return_detail, a dict
    with the continuous column u_c, the elevation phi and the number of
    fixed-point steps taken.
    """
    X = np.asarray(X, np.float64)
    shp = X.shape[:-1]
    X = X.reshape(-1, 3)
    phi_lut = np.asarray(phi_lut, np.float64)
    theta_lut = np.asarray(theta_lut, np.float64)
    x, y, z = X[:, 0], X[:, 1], X[:, 2]

    def one_pass(uc):
        col = TWO_PI * uc / W
        xp = x - r0 * np.cos(col)
        yp = y - r0 * np.sin(col)
        r = np.sqrt(xp * xp + yp * yp + z * z)
        with np.errstate(invalid="ignore", divide="ignore"):
            phi = np.arcsin(np.clip(z / r, -1.0, 1.0))
        phi_safe = np.where(np.isfinite(phi), phi, 0.0)
        v = row_argmin(phi_safe, phi_lut)
        theta = np.mod(np.arctan2(yp, xp), TWO_PI)
        u_hat = W * theta / TWO_PI
        uc_new = u_hat - W * theta_lut[v] / TWO_PI
        return uc_new, v, r, phi

    # start: the column angle from atan2(y, x), offset-free
    uc = W * np.mod(np.arctan2(y, x), TWO_PI) / TWO_PI
    steps = 0
    if r0 != 0.0:
        for steps in range(1, max_iter + 1):
            uc_new, v, r, phi = one_pass(uc)
            # compare the column angles modulo W
            du = np.abs(np.mod(uc_new - uc + 0.5 * W, W) - 0.5 * W)
            uc = uc_new
            if np.all(du[np.isfinite(du)] < tol):
                break
    uc, v, r, phi = one_pass(uc)
    lo, hi = fov_limits(phi_lut)
    in_fov = np.isfinite(phi) & (phi >= lo) & (phi <= hi) & (r > 0)
    uc_safe = np.where(np.isfinite(uc), uc, 0.0)
    u = np.mod(np.floor(uc_safe + 0.5).astype(np.int64), W)
    out = (u.reshape(shp), v.reshape(shp), r.reshape(shp), in_fov.reshape(shp))
    if return_detail:
        return out + (dict(u_c=uc.reshape(shp), phi=phi.reshape(shp), steps=steps),)
    return out


def inverse_lut_build(phi_lut, n_bins=None):
    """The inverse elevation table of Section 3.2: n_bins (default 2H) uniform
    bins over [min phi_lut, max phi_lut]; each bin stores the row nearest to
    the bin centre.  Returns (table, phi0, bin_width)."""
    phi_lut = np.asarray(phi_lut, np.float64)
    H = phi_lut.shape[0]
    n_bins = 2 * H if n_bins is None else n_bins
    lo, hi = phi_lut.min(), phi_lut.max()
    width = (hi - lo) / n_bins
    centres = lo + (np.arange(n_bins) + 0.5) * width
    return row_argmin(centres, phi_lut), lo, width


def inverse_lut_row(phi, table, phi0, width):
    """Candidate row from the inverse table (bin lookup only, no refinement)."""
    b = np.floor((np.asarray(phi, np.float64) - phi0) / width).astype(np.int64)
    return table[np.clip(b, 0, table.shape[0] - 1)]


def inverse_lut_refined(phi, phi_lut, table, phi0, width):
    """Candidate row refined over its +-1 neighbours by the Eq. 4 distance
    (ties -> lower row index)."""
    phi = np.asarray(phi, np.float64)
    c = inverse_lut_row(phi, table, phi0, width)
    H = phi_lut.shape[0]
    best = c.copy()
    bestd = np.abs(phi_lut[c] - phi)
    for off in (-1, 1):
        t = np.clip(c + off, 0, H - 1)
        d = np.abs(phi_lut[t] - phi)
        better = (d < bestd) | ((d == bestd) & (t < best))
        best = np.where(better, t, best)
        bestd = np.where(better, d, bestd)
    return best


# ----------------------------------------------------------------------------
# Section 4.1: strided pyramid and neighbour normals

def pyramid(img, levels):
    """Level l = the image strided by 2^l in rows and columns (Section 4.1)."""
    img = np.asarray(img)
    return [img[:: 1 << l, :: 1 << l] for l in range(levels)]


def normals(range_img, phi_lut, theta_lut, r0, rel_jump, return_margin=False):
    """Normal image from the cross product of neighbouring pixels' points.

    Returns n (H, W, 3) float64 (zero where invalid) and the validity mask; with
    return_margin also the relative distance of the degeneracy test to its
    threshold (for near-tie flagging)."""
    rimg = np.asarray(range_img, np.float64)
    H, W = rimg.shape
    P, valid = unproject(rimg, phi_lut, theta_lut, r0)
    r = np.where(valid, rimg, 0.0)
    jump = np.float64(rel_jump)
    left, right = np.roll(P, 1, axis=1), np.roll(P, -1, axis=1)      # u-1, u+1 (wrap)
    rl, rr = np.roll(r, 1, axis=1), np.roll(r, -1, axis=1)
    vl, vr = np.roll(valid, 1, axis=1), np.roll(valid, -1, axis=1)
    up = np.zeros_like(P); down = np.zeros_like(P)
    ru = np.zeros_like(r); rd = np.zeros_like(r)
    vu = np.zeros_like(valid); vd = np.zeros_like(valid)
    up[1:] = P[:-1]; ru[1:] = r[:-1]; vu[1:] = valid[:-1]              # v-1
    down[:-1] = P[1:]; rd[:-1] = r[1:]; vd[:-1] = valid[1:]            # v+1
    a = right - left
    b = down - up
    c = np.cross(a, b)
    cn = np.linalg.norm(c, axis=-1)
    an = np.linalg.norm(a, axis=-1)
    bn = np.linalg.norm(b, axis=-1)
    ok = valid & vl & vr & vu & vd
    for rn in (rl, rr, ru, rd):
        ok &= np.abs(rn - r) <= jump * r
    rows = np.zeros((H, 1), bool)
    rows[1:H - 1] = True
    ok &= rows
    thr = NORMAL_SIN_EPS * an * bn
    ok &= cn > thr
    with np.errstate(invalid="ignore", divide="ignore"):
        n = c / cn[..., None]
    flip = np.sum(n * P, axis=-1) > 0
    n = np.where(flip[..., None], -n, n)
    n = np.where(ok[..., None], n, 0.0)
    if return_margin:
        with np.errstate(invalid="ignore", divide="ignore"):
            margin = np.where(thr > 0, np.abs(cn - thr) / thr, np.inf)
        return n, ok, margin
    return n, ok


PCA_MIN_POINTS = 5          # points of the 3x3 window needed for a PCA normal
PCA_COLLINEAR = 1e-4        # lambda_1 <= this * lambda_2: the window's points lie on a line


def normals_pca(range_img, phi_lut, theta_lut, r0, rel_jump, return_detail=False):
    """Normal image by eigen-decomposition of the 3x3 pixel window (the
    alternative Section 4.1 names beside the cross product).

    The window of pixel (u, v) holds the valid points of rows v-1 .. v+1 and
    columns u-1 .. u+1 (u wraps) whose range differs from the centre's by at
    most rel_jump times the centre's range.  With k >= PCA_MIN_POINTS such
    points (the centre included), the normal is the eigenvector of the
    smallest eigenvalue of their scatter matrix sum (p - mean)(p - mean)^T,
    oriented so that n . P <= 0 (P the centre point); the plane offset of the
    library's plane image is then n . P.  Invalid on rows 0 and H-1, at an
    invalid centre, with fewer points, or when lambda_1 <= PCA_COLLINEAR *
    lambda_2 (collinear points leave the normal undetermined).

    Returns n (H, W, 3) (zero where invalid) and the validity mask; with
    return_detail also the eigenvalues (H, W, 3) ascending, the point count
    and the relative distance of the collinearity test to its threshold."""
    rimg = np.asarray(range_img, np.float64)
    H, W = rimg.shape
    P, valid = unproject(rimg, phi_lut, theta_lut, r0)
    r = np.where(valid, rimg, 0.0)
    pts = np.zeros((H, W, 9, 3))
    use = np.zeros((H, W, 9), bool)
    k = 0
    for dv in (-1, 0, 1):
        for du in (-1, 0, 1):
            Pn = np.zeros_like(P)
            rn = np.zeros_like(r)
            vn = np.zeros_like(valid)
            src_rows = slice(max(0, dv), H + min(0, dv))
            dst_rows = slice(max(0, -dv), H + min(0, -dv))
            Pn[dst_rows] = np.roll(P, -du, axis=1)[src_rows]
            rn[dst_rows] = np.roll(r, -du, axis=1)[src_rows]
            vn[dst_rows] = np.roll(valid, -du, axis=1)[src_rows]
            pts[:, :, k] = Pn
            use[:, :, k] = vn & valid & (np.abs(rn - r) <= rel_jump * r)
            k += 1
    cnt = use.sum(axis=-1)
    w = use[..., None].astype(np.float64)
    mean = (pts * w).sum(axis=2) / np.maximum(cnt, 1)[..., None]
    q = (pts - mean[:, :, None, :]) * w
    C = np.einsum("hwki,hwkj->hwij", q, q)
    lam, vec = np.linalg.eigh(C.reshape(-1, 3, 3))
    lam = lam.reshape(H, W, 3)
    n = vec[:, :, 0].reshape(H, W, 3)
    rows = np.zeros((H, 1), bool)
    rows[1:H - 1] = True
    thr = PCA_COLLINEAR * lam[..., 2]
    ok = valid & rows & (cnt >= PCA_MIN_POINTS) & (lam[..., 1] > thr)
    flip = np.sum(n * P, axis=-1) > 0
    n = np.where(flip[..., None], -n, n)
    n = np.where(ok[..., None], n, 0.0)
    if return_detail:
        with np.errstate(invalid="ignore", divide="ignore"):
            margin = np.where(thr > 0, np.abs(lam[..., 1] - thr) / thr, np.inf)
        return n, ok, dict(lam=lam, count=cnt, margin=margin)
    return n, ok


# ----------------------------------------------------------------------------
# Section 4.1: projective association (Eq. 5-6), point-to-plane loss and
# the Gauss-Newton normal equations of Eq. 7

H21 = [(i, j) for i in range(6) for j in range(i, 6)]   # upper triangle, row-major


def icp_terms(P_src, src_valid, T, dst_range, dst_n, dst_nvalid, phi_l, theta_l, r0,
              huber_delta, max_corr_dist=0.0, dst_n_margin=None, assoc=None):
    """Associate every source point with the target image and build the
    weighted normal equations at pose T.

    assoc (optional, int per source point, v*W+u or -1): use these
    associations instead of deciding them by the projection (every other
    step unchanged).  This isolates the arithmetic of a step from its
    discrete decisions when checking an implementation that decided a few
    near-tie pixels the other way.

    Returns dict with H (6x6), g (6), sum_wr2, count, assoc (int64 index
    v*W+u or -1 per source point), near_tie (bool per source point), the
    per-point residual e, weight w and Jacobian J (0 where not associated),
    and the two distances the near-tie flag is read from: margin_u, the
    distance of the continuous column u_c to the nearest half-integer (the
    rounding boundary of the column choice, in pixels), and margin_row, the
    distance of the elevation to the nearest row boundary or field-of-view
    edge in units of the local row spacing (row_margin)."""
    P = np.asarray(P_src, np.float64).reshape(-1, 3)
    sv = np.asarray(src_valid, bool).reshape(-1)
    T = np.asarray(T, np.float64)
    R, t = T[:3, :3], T[:3, 3]
    Hh, Wd = dst_range.shape
    X = P @ R.T + t                                             # R_k p + t_k
    u, v, _, in_fov, det = project(X, phi_l, theta_l, r0, Wd, return_detail=True)   # Eq. 5
    if assoc is not None:
        a = np.asarray(assoc, np.int64).reshape(-1)
        in_fov = a >= 0
        v = np.where(in_fov, a // Wd, 0)
        u = np.where(in_fov, a % Wd, 0)
    rq = np.asarray(dst_range, np.float64)[v, u]
    q = unproject_pixels(u, v, np.where(range_valid(rq), rq, 0.0), phi_l, theta_l, r0, Wd)  # Eq. 6
    n = np.asarray(dst_n, np.float64)[v, u]
    ok = sv & in_fov & range_valid(rq) & np.asarray(dst_nvalid, bool)[v, u]
    diff = X - q
    dist = np.linalg.norm(diff, axis=-1)
    if max_corr_dist > 0:
        ok &= dist <= max_corr_dist
    e = np.sum(n * diff, axis=-1)                               # n_q^T (x - q)
    if huber_delta > 0:
        w = 1.0 / np.sqrt(1.0 + (e / huber_delta) ** 2)         # pseudo-Huber IRLS weight
    else:
        w = np.ones_like(e)
    w = np.where(ok, w, 0.0)
    e = np.where(ok, e, 0.0)
    J = np.concatenate([np.cross(X, n), n], axis=-1)            # d e / d (omega, tau)
    J = np.where(ok[:, None], J, 0.0)
    Hm = (J * w[:, None]).T @ J
    g = (J * (w * e)[:, None]).sum(axis=0)
    # near-tie flags: decisions an FP32 implementation may legitimately take
    # the other way
    uc = det["u_c"]
    with np.errstate(invalid="ignore"):
        m_u = np.abs(uc - (np.floor(uc) + 0.5))
    m_v = row_margin(np.where(np.isfinite(det["phi"]), det["phi"], 0.0), phi_l)
    near = sv & ((m_u < NEAR_TIE_PX) | (m_v < NEAR_TIE_ROW))
    if dst_n_margin is not None:
        near |= sv & in_fov & (np.asarray(dst_n_margin)[v, u] < 1e-3)
    if max_corr_dist > 0:
        near |= sv & in_fov & (np.abs(dist - max_corr_dist) < 1e-5 * max_corr_dist)
    assoc = np.where(ok, v * Wd + u, -1)
    return dict(H=Hm, g=g, sum_wr2=float(np.sum(w * e * e)), count=int(ok.sum()),
                assoc=assoc, near_tie=near, margin_u=m_u, margin_row=m_v, e=e, w=w, X=X, J=J)


def pack29(terms):
    """The 29 reduced quantities in the library's order: 21 upper-triangle
    entries of J^T W J (row-major), 6 of J^T W e, sum w e^2, count."""
    Hm, g = terms["H"], terms["g"]
    return np.array([Hm[i, j] for i, j in H21] + list(g) + [terms["sum_wr2"], terms["count"]],
                    np.float64)


def cholesky_solve(Hm, g):
    """Solve Hm x = -g by a textbook LL^T factorisation.  Returns (x, ok); ok is
    False when a pivot is <= 1e-12 * trace(Hm) (x is then zero)."""
    n = Hm.shape[0]
    L = np.zeros((n, n))
    tr = np.trace(Hm)
    for j in range(n):
        d = Hm[j, j] - sum(L[j, k] ** 2 for k in range(j))
        if not (d > CHOL_REL_EPS * tr):
            return np.zeros(n), False
        L[j, j] = np.sqrt(d)
        for i in range(j + 1, n):
            L[i, j] = (Hm[i, j] - sum(L[i, k] * L[j, k] for k in range(j))) / L[j, j]
    y = np.zeros(n)
    for i in range(n):
        y[i] = (-g[i] - sum(L[i, k] * y[k] for k in range(i))) / L[i, i]
    x = np.zeros(n)
    for i in reversed(range(n)):
        x[i] = (y[i] - sum(L[k, i] * x[k] for k in range(i + 1, n))) / L[i, i]
    return x, True


def hat(w):
    return np.array([[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]], np.float64)


def se3_exp(xi):
    """Exp of a twist xi = (omega, tau): Rodrigues rotation and the V matrix;
    second-order series below 1e-8 rad."""
    w = np.asarray(xi[:3], np.float64)
    tau = np.asarray(xi[3:], np.float64)
    th = np.linalg.norm(w)
    K = hat(w)
    K2 = K @ K
    if th < 1e-8:
        A, B, C = 1.0 - th * th / 6.0, 0.5 - th * th / 24.0, 1.0 / 6.0 - th * th / 120.0
    else:
        A = np.sin(th) / th
        B = (1.0 - np.cos(th)) / (th * th)
        C = (th - np.sin(th)) / (th ** 3)
    Rm = np.eye(3) + A * K + B * K2
    V = np.eye(3) + B * K + C * K2
    T = np.eye(4)
    T[:3, :3] = Rm
    T[:3, 3] = V @ tau
    return T


def gn_update(T, terms):
    """One Gauss-Newton update T <- Exp(xi) T from the normal equations.
    Returns (T_new, ok)."""
    if terms["count"] < 6:
        return np.array(T, np.float64), False
    xi, ok = cholesky_solve(terms["H"], terms["g"])
    if not ok:
        return np.array(T, np.float64), False
    return se3_exp(xi) @ T, True


class Target:
    """A target scan prepared for association: range pyramid plus strided
    normal images (Section 4.1)."""

    def __init__(self, dst_range, phi_lut, theta_lut, r0, levels, rel_jump, normal_method="cross"):
        self.phi, self.theta, self.r0 = np.asarray(phi_lut, np.float64), np.asarray(theta_lut, np.float64), float(r0)
        if normal_method == "pca":
            n0, ok0, det = normals_pca(dst_range, self.phi, self.theta, self.r0, rel_jump, return_detail=True)
            m0 = det["margin"]
        else:
            n0, ok0, m0 = normals(dst_range, self.phi, self.theta, self.r0, rel_jump, return_margin=True)
        self.range = pyramid(np.asarray(dst_range), levels)
        self.n = pyramid(n0, levels)
        self.nvalid = pyramid(ok0, levels)
        self.nmargin = pyramid(m0, levels)

    def level(self, l):
        ph, th = level_tables(self.phi, self.theta, l)
        return self.range[l], self.n[l], self.nvalid[l], ph, th


def source_points(src_range, phi_lut, theta_lut, r0, level):
    """Source points of level l: unprojection of the strided range image with
    the strided tables (equal to the finest-level points at (2^l u, 2^l v))."""
    ph, th = level_tables(phi_lut, theta_lut, level)
    s = 1 << level
    return unproject(np.asarray(src_range)[::s, ::s], ph, th, r0)


def icp_step(src_pts, src_valid, target, level, T, params):
    """One association + Gauss-Newton step at a pyramid level."""
    rng_l, n_l, nv_l, ph, th = target.level(level)
    terms = icp_terms(src_pts, src_valid, T, rng_l, n_l, nv_l, ph, th, target.r0,
                      params.get("huber_delta", 0.5), params.get("max_corr_dist", 0.0),
                      dst_n_margin=target.nmargin[level])
    T_new, ok = gn_update(T, terms)
    return T_new, ok, terms


def register(src_range, dst_range, src_sensor, dst_sensor, T_init, levels, iters, params,
             return_history=False, return_poses=False):
    """Multi-scale registration: for each level from coarsest to finest run
    the scheduled number of Gauss-Newton steps; the pose carries over between
    levels unchanged.  ``iters`` is listed coarse -> fine.  Sensors are
    (phi_lut, theta_lut, r0) tuples.  return_history adds every step's
    record (poses and terms); return_poses adds only the list of the poses
    after each step (the initial pose first)."""
    assert len(iters) == levels
    sp, st, sr0 = src_sensor
    target = Target(dst_range, *dst_sensor, levels, params.get("normal_rel_jump", np.float32(0.1)),
                    params.get("normal_method", "cross"))
    T = np.array(T_init, np.float64)
    degenerate = False
    hist = []
    poses = [T]
    for k, l in enumerate(range(levels - 1, -1, -1)):
        P, sv = source_points(src_range, sp, st, sr0, l)
        for _ in range(iters[k]):
            T_prev = T
            T, ok, terms = icp_step(P, sv, target, l, T, params)
            degenerate |= not ok
            if return_history:
                hist.append(dict(level=l, T_in=T_prev, T_out=T, terms=terms, ok=ok))
            if return_poses:
                poses.append(T)
    if return_history:
        return T, degenerate, hist
    if return_poses:
        return T, degenerate, poses
    return T, degenerate


def center_align(P_src, P_dst):
    """Initial pose of the registration problem (Section 4.1: the rotation
    starts at the identity and the translation aligns the centres of the two
    point sets): R = I, t = mean(P_dst) - mean(P_src), so that x = p + t maps
    the source centre onto the target centre.  Either set empty: identity."""
    P_src = np.asarray(P_src, np.float64).reshape(-1, 3)
    P_dst = np.asarray(P_dst, np.float64).reshape(-1, 3)
    T = np.eye(4)
    if len(P_src) and len(P_dst):
        T[:3, 3] = P_dst.mean(axis=0) - P_src.mean(axis=0)
    return T


def center_init(src_range, dst_range, src_sensor, dst_sensor, level=0):
    """center_align of the valid points of two range images at pyramid level
    l (Eq. 1-2 on the strided images, Section 4.1).  Sensors are (phi_lut,
    theta_lut, r0) tuples.  Returns (T, ok); ok is False (T = I) when either
    image has no valid pixel."""
    P_s, v_s = source_points(src_range, *src_sensor, level)
    P_d, v_d = source_points(dst_range, *dst_sensor, level)
    return center_align(P_s[v_s], P_d[v_d]), bool(v_s.any() and v_d.any())


def pose_error(T, T_ref):
    """Rotation error arccos((tr(R R_ref^T) - 1) / 2) in radians and translation
    error |t - t_ref| in metres (the evaluation metric of Section 6.1, read with
    the trace and without the square)."""
    R, Rr = np.asarray(T)[:3, :3], np.asarray(T_ref)[:3, :3]
    c = np.clip((np.trace(R @ Rr.T) - 1.0) / 2.0, -1.0, 1.0)
    return float(np.arccos(c)), float(np.linalg.norm(np.asarray(T)[:3, 3] - np.asarray(T_ref)[:3, 3]))


# ----------------------------------------------------------------------------
# Point clouds without scan structure (Section 3.2, last paragraph): projected
# into a range image through Pi; each pixel keeps its nearest point.

def points_to_range(X, phi_lut, theta_lut, r0, W):
    """Range image [H, W] of points X (n, 3) (already in the sensor frame):
    pixel (u, v) = Pi(x) holds the smallest range r of the points projecting
    there inside the vertical field of view; pixels without points hold +inf.
    Also returns a mask of pixels that a near-tie point (within NEAR_TIE_PX
    of a column boundary or NEAR_TIE_ROW of a row boundary) could have
    reached: the pixel it was given and its 8 neighbours (columns wrap)."""
    X = np.asarray(X, np.float64).reshape(-1, 3)
    H = len(phi_lut)
    ok = np.all(np.isfinite(X), axis=1)
    Xs = np.where(ok[:, None], X, 1.0)
    u, v, r, fov, det = project(Xs, phi_lut, theta_lut, r0, W, return_detail=True)
    keep = ok & fov & (r > 0)
    img = np.full((H, W), np.inf)
    np.minimum.at(img, (v[keep], u[keep]), r[keep])
    m_u = np.abs(np.mod(det["u_c"], 1.0) - 0.5)
    m_v = row_margin(np.where(np.isfinite(det["phi"]), det["phi"], 0.0), phi_lut)
    near_pt = ok & ((m_u < NEAR_TIE_PX) | (m_v < NEAR_TIE_ROW)) & (r > 0)
    near = np.zeros((H, W), bool)
    for dv in (-1, 0, 1):
        for du in (-1, 0, 1):
            vv = np.clip(v[near_pt] + dv, 0, H - 1)
            near[vv, np.mod(u[near_pt] + du, W)] = True
    return img, near
