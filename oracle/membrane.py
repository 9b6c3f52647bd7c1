"""Overset finite-difference surface derivatives and the Skalak membrane force,
written out plainly in FP64 NumPy.

This is test infrastructure: only the tests, the smoke check and the bench's
CPU baseline use it; the library never does, and it shares no code with the
CUDA path. It takes the steps of Sec. 3.5 (surface derivatives) in the
paper's order and notation (arXiv 2310.13908):

  * transition maps tau_ij = (eta_j^0)^{-1} o eta_i^0 ........ Sec. 3.1, Appendix
  * patch extension to the ghost grid, Eq. ext (cont. Eq. cont_ext)
  * 7-point central finite differences on the extended grid, Eq. fdm
  * blending with the transition Jacobians, Eqs. blendu / blendv
  * E, F, G, W, n, L, M, N, H, K and the surface divergence . Appendix, Table diff_formulas
  * Skalak tension Lambda .................................... Sec. 2.1, Eq. tensor
  * membrane force f = div_gamma Lambda ...................... Sec. 2.1, Eq. intf
  * area and volume (V = int (x, 0, 0) . n) .................. Sec. 4.1

Readings (the paper is silent or misprinted):
  * "cubic splines interpolation" I_ij: the tensor-product not-a-knot cubic
    spline on patch j's (m-1) x (m-1) grid, continued by its end pieces
    outside the node range.
  * The 7-point stencil is the standard central first-derivative stencil
    (-1, 9, -45, 0, 45, -9, 1) / 60h; the paper calls it fifth order in one
    place and fourth in another.
  * The transition maps are computed as the chart composition that defines
    them (Sec. 3.1). It agrees with the Appendix's formulas except for two
    misprints: tau_56 and tau_65 are printed as (pi - u, v) (the composition
    gives (pi - u, -v)), and tau_63, tau_64 carry the opposite sign of cos u.
  * Second fundamental form (for H and K): from the derivatives of the
    Cartesian normal field, L = -x_u . n_u etc. (x_u is not a function on
    the surface, so it cannot go through the patch extension).
"""

from __future__ import annotations

import numpy as np
from scipy.interpolate import CubicSpline

from capsule_inputs.geometry import chart, chart_tangents, pou_all

# central first-derivative stencil on offsets -3..3 (times 1/h)
FD7 = np.array([-1.0, 9.0, -45.0, 0.0, 45.0, -9.0, 1.0]) / 60.0
GHOST = 3  # ghost layers on each side of a patch grid


def inverse_chart(p: int, x0: np.ndarray):
    """(eta_p^0)^{-1}: the (u, v) of unit vectors x0 in patch p (Eq. param_maps).

    u = arccos of the chart's cos-u component, v = atan2 of its sin-u sin-v and
    sin-u cos-v components; inside the patch (0 < v < pi) this is the inverse.
    """
    x, y, z = x0[..., 0], x0[..., 1], x0[..., 2]
    if p == 1:
        cu, a, b = z, x, y
    elif p == 2:
        cu, a, b = z, -x, -y
    elif p == 3:
        cu, a, b = z, -y, x
    elif p == 4:
        cu, a, b = z, y, -x
    elif p == 5:
        cu, a, b = -y, x, z
    elif p == 6:
        cu, a, b = y, x, -z
    else:
        raise ValueError(p)
    return np.arccos(np.clip(cu, -1.0, 1.0)), np.arctan2(b, a)


def transition(i: int, j: int, u, v):
    """tau_ij(u, v) = (eta_j^0)^{-1}(eta_i^0(u, v)) (Sec. 3.1)."""
    return inverse_chart(j, chart(i, u, v))


def transition_jacobian(i: int, j: int, u, v):
    """Jacobian of tau_ij as laid out in Eq. jacobian_diff:
    [[d tau1/du, d tau2/du], [d tau1/dv, d tau2/dv]], shape (..., 2, 2).

    By the chain rule the tangents of chart i are combinations of those of
    chart j at the same point: eta_i,u = eta_j,u' dtau1/du + eta_j,v' dtau2/du
    (and the same for v); solved by least squares (the system is consistent).
    """
    ti_u, ti_v = chart_tangents(i, u, v)
    uj, vj = transition(i, j, u, v)
    tj_u, tj_v = chart_tangents(j, uj, vj)
    A = np.stack([tj_u, tj_v], axis=-1)                     # (..., 3, 2)
    rhs = np.stack([ti_u, ti_v], axis=-1)                   # (..., 3, 2)
    sol = np.linalg.solve(np.swapaxes(A, -1, -2) @ A, np.swapaxes(A, -1, -2) @ rhs)
    # sol[..., :, 0] = (dtau1/du, dtau2/du), sol[..., :, 1] = (dtau1/dv, dtau2/dv)
    return np.swapaxes(sol, -1, -2)


def nodes(m: int) -> np.ndarray:
    """Grid coordinates j pi / m, j = 1..m-1 (Sec. 3.2)."""
    return np.arange(1, m) * np.pi / m


def spline_weights(m: int, t) -> np.ndarray:
    """Cardinal weights of the not-a-knot cubic spline through the m-1 grid
    nodes, evaluated at t (continued by the end pieces): shape (len(t), m-1)."""
    t = np.atleast_1d(np.asarray(t, dtype=np.float64))
    cs = CubicSpline(nodes(m), np.eye(m - 1), bc_type="not-a-knot", extrapolate=True)
    return cs(t)


def interpolate(m: int, Gp: np.ndarray, u, v) -> np.ndarray:
    """I_ij: the tensor-product cubic spline of one patch's grid values
    Gp[(m-1), (m-1), F] at the points (u, v); returns (len(u), F)."""
    Wu = spline_weights(m, u)
    Wv = spline_weights(m, v)
    return np.einsum("na,abf,nb->nf", Wu, Gp, Wv)


def _as_patches(m: int, G: np.ndarray) -> np.ndarray:
    n = m - 1
    G = np.asarray(G, dtype=np.float64)
    return G.reshape(6, n, n, -1)


def extend(m: int, G: np.ndarray) -> np.ndarray:
    """Patch extension, Eq. ext: values on the extended grids
    (j, k = -2..m+2), shape (6, m+5, m+5, F). Interior nodes keep their values;
    a ghost point x1 = eta_i^0(u1, v1) gets sum_j psi_j(x1) I_ij(g^j)(tau_ij).
    Only ghost points with one index inside 1..m-1 (those the stencils use)
    are filled; the corner blocks stay NaN."""
    Gp = _as_patches(m, G)
    n, F = m - 1, Gp.shape[-1]
    h = np.pi / m
    ext = np.full((6, m + 5, m + 5, F), np.nan)
    idx = np.arange(-2, m + 3)                       # extended index j
    inner = (idx >= 1) & (idx <= m - 1)
    for i in range(1, 7):
        ext[i - 1][np.ix_(inner, inner)] = Gp[i - 1]
        jj, kk = np.meshgrid(idx, idx, indexing="ij")
        ghost = (~inner[:, None] & inner[None, :]) | (inner[:, None] & ~inner[None, :])
        gj, gk = jj[ghost], kk[ghost]
        x1 = chart(i, gj * h, gk * h)
        psi = pou_all(x1)                             # (P, 6)
        val = np.zeros((len(gj), F))
        for p in range(1, 7):
            sel = psi[:, p - 1] > 0.0
            if not np.any(sel):
                continue
            up, vp = inverse_chart(p, x1[sel])
            val[sel] += psi[sel, p - 1][:, None] * interpolate(m, Gp[p - 1], up, vp)
        ext[i - 1][ghost] = val
    return ext


def finite_differences(m: int, ext: np.ndarray):
    """Eq. fdm: central 7-point u- and v-derivatives at the grid nodes of every
    patch from the extended values; returns two (6, m-1, m-1, F) arrays."""
    h = np.pi / m
    n = m - 1
    du = np.zeros((6, n, n, ext.shape[-1]))
    dv = np.zeros_like(du)
    for s, c in zip(range(-3, 4), FD7):
        if c == 0.0:
            continue
        # node j (1..m-1) sits at extended index j + 2
        du += c * ext[:, 3 + s:3 + s + n, 3:3 + n]
        dv += c * ext[:, 3:3 + n, 3 + s:3 + s + n]
    return du / h, dv / h


def blend(m: int, du: np.ndarray, dv: np.ndarray):
    """Eqs. blendu / blendv: at every node of patch i,
    g_u = psi_i g_u^i + sum_{j != i} psi_j (I_ij(g_u^j) dtau1/du + I_ij(g_v^j) dtau2/du),
    g_v likewise with the v-derivatives of tau_ij; psi at the node."""
    n = m - 1
    h = np.pi / m
    F = du.shape[-1]
    j_, k_ = np.meshgrid(np.arange(1, m), np.arange(1, m), indexing="ij")
    u, v = (j_ * h).ravel(), (k_ * h).ravel()
    out_u = np.zeros((6, n * n, F))
    out_v = np.zeros_like(out_u)
    for i in range(1, 7):
        x0 = chart(i, u, v)
        psi = pou_all(x0)
        out_u[i - 1] = psi[:, i - 1, None] * du[i - 1].reshape(-1, F)
        out_v[i - 1] = psi[:, i - 1, None] * dv[i - 1].reshape(-1, F)
        for p in range(1, 7):
            if p == i:
                continue
            sel = psi[:, p - 1] > 0.0
            if not np.any(sel):
                continue
            up, vp = transition(i, p, u[sel], v[sel])
            Iu = interpolate(m, du[p - 1], up, vp)
            Iv = interpolate(m, dv[p - 1], up, vp)
            J = transition_jacobian(i, p, u[sel], v[sel])
            w = psi[sel, p - 1][:, None]
            out_u[i - 1, sel] += w * (Iu * J[:, 0, 0, None] + Iv * J[:, 0, 1, None])
            out_v[i - 1, sel] += w * (Iu * J[:, 1, 0, None] + Iv * J[:, 1, 1, None])
    return out_u.reshape(6 * n * n, F), out_v.reshape(6 * n * n, F)


def surface_derivatives(m: int, G: np.ndarray, blending: bool = True):
    """u- and v-derivatives of node values G (N, F) by extension, finite
    differences and (optionally) blending (Sec. 3.5); returns (Gu, Gv)."""
    G = np.asarray(G, dtype=np.float64)
    flat = G.reshape(G.shape[0], -1)
    du, dv = finite_differences(m, extend(m, flat))
    if blending:
        gu, gv = blend(m, du, dv)
    else:
        gu, gv = du.reshape(flat.shape), dv.reshape(flat.shape)
    return gu.reshape(G.shape), gv.reshape(G.shape)


def first_form(xu: np.ndarray, xv: np.ndarray):
    """E, F, G, W and n = x_u x x_v / W (Appendix, Table diff_formulas)."""
    E = np.sum(xu * xu, axis=-1)
    F = np.sum(xu * xv, axis=-1)
    G = np.sum(xv * xv, axis=-1)
    W = np.sqrt(E * G - F * F)
    n = np.cross(xu, xv) / W[:, None]
    return E, F, G, W, n


def geometry(m: int, X: np.ndarray, blending: bool = True) -> dict:
    """Tangents, first fundamental form, area element and normals of nodes X."""
    xu, xv = surface_derivatives(m, X, blending)
    E, F, G, W, n = first_form(xu, xv)
    return {"xu": xu, "xv": xv, "E": E, "F": F, "G": G, "W": W, "n": n}


def curvatures(m: int, X: np.ndarray, blending: bool = True):
    """Mean and Gaussian curvature H = (EN - 2FM + GL) / (2W^2),
    K = (LN - M^2) / W^2 (Appendix, Table diff_formulas).

    The scheme of Sec. 3.5 differentiates functions on the surface; x_u is not
    one (it depends on the patch's parameterization), the Cartesian normal n
    is. So L = x_uu.n = -x_u.n_u, M = -x_u.n_v, N = -x_v.n_v (from x_u.n = 0),
    with n_u, n_v by the scheme.
    """
    g = geometry(m, X, blending)
    nu, nv = surface_derivatives(m, g["n"], blending)
    L = -np.sum(g["xu"] * nu, axis=-1)
    M = -np.sum(g["xu"] * nv, axis=-1)
    N = -np.sum(g["xv"] * nv, axis=-1)
    E, F, G, W = g["E"], g["F"], g["G"], g["W"]
    H = (E * N - 2 * F * M + G * L) / (2 * W * W)
    K = (L * N - M * M) / (W * W)
    return H, K


def divergence_from(geo: dict, gu: np.ndarray, gv: np.ndarray) -> np.ndarray:
    """div_gamma g = (G g_u - F g_v)/W^2 . x_u + (E g_v - F g_u)/W^2 . x_v
    (Appendix, Table diff_formulas), for vector fields g (..., 3)."""
    E, F, G, W = geo["E"], geo["F"], geo["G"], geo["W"]
    W2 = (W * W)[:, None]
    a = (G[:, None] * gu - F[:, None] * gv) / W2
    b = (E[:, None] * gv - F[:, None] * gu) / W2
    return np.sum(a * geo["xu"], axis=-1) + np.sum(b * geo["xv"], axis=-1)


def surface_divergence(m: int, X: np.ndarray, g: np.ndarray) -> np.ndarray:
    """div_gamma of a vector field g given at the nodes X."""
    geo = geometry(m, X)
    gu, gv = surface_derivatives(m, g)
    return divergence_from(geo, gu, gv)


def skalak_tension(geo: dict, ref: dict, Es: float, ED: float) -> np.ndarray:
    """Lambda of Eq. tensor at every node, shape (N, 3, 3).

    F_s maps the reference tangents to the current ones and the reference
    normal to 0 (Sec. 2.1): F_s = [a1 a2 0] [a1r a2r nr]^{-1}; V^2 = F_s F_s^T,
    lambda_1^2, lambda_2^2 its two nonzero eigenvalues, I1 = l1^2 + l2^2 - 2,
    I2 = l1^2 l2^2 - 1, J_s = l1 l2, P = I - n n^T, and
    Lambda = Es/(2 J_s) (I1 + 1) V^2 + J_s/2 (ED I2 - Es) P.
    """
    N = geo["xu"].shape[0]
    A = np.stack([ref["xu"], ref["xv"], ref["n"]], axis=-1)        # columns
    B = np.stack([geo["xu"], geo["xv"], np.zeros((N, 3))], axis=-1)
    Fs = B @ np.linalg.inv(A)
    V2 = Fs @ np.swapaxes(Fs, -1, -2)
    ev = np.sort(np.linalg.eigvalsh(V2), axis=-1)[:, 1:]            # two nonzero
    l1s, l2s = ev[:, 0], ev[:, 1]
    I1 = l1s + l2s - 2.0
    I2 = l1s * l2s - 1.0
    Js = np.sqrt(l1s * l2s)
    n = geo["n"]
    P = np.eye(3)[None] - n[:, :, None] * n[:, None, :]
    return ((Es / (2.0 * Js) * (I1 + 1.0))[:, None, None] * V2
            + (0.5 * Js * (ED * I2 - Es))[:, None, None] * P)


def skalak_force(m: int, X: np.ndarray, X_ref: np.ndarray, Es: float, ED: float) -> np.ndarray:
    """f = div_gamma Lambda (Eq. intf) at the nodes X: the divergence of each
    column Lambda[:, k] (Lambda is symmetric), with every derivative by the
    scheme of Sec. 3.5; reference tangents from X_ref by the same scheme."""
    geo = geometry(m, X)
    ref = geometry(m, X_ref)
    Lam = skalak_tension(geo, ref, Es, ED)
    Lu, Lv = surface_derivatives(m, Lam.reshape(-1, 9))
    Lu = Lu.reshape(-1, 3, 3)
    Lv = Lv.reshape(-1, 3, 3)
    f = np.empty((X.shape[0], 3))
    for k in range(3):
        f[:, k] = divergence_from(geo, Lu[:, :, k], Lv[:, :, k])
    return f


def pou_weights(m: int) -> np.ndarray:
    """psi of each node's own patch (Eq. pou), node order of the grid."""
    n = m - 1
    h = np.pi / m
    j_, k_ = np.meshgrid(np.arange(1, m), np.arange(1, m), indexing="ij")
    u, v = (j_ * h).ravel(), (k_ * h).ravel()
    out = np.empty((6, n * n))
    for i in range(1, 7):
        out[i - 1] = pou_all(chart(i, u, v))[:, i - 1]
    return out.ravel()


def quadrature_weights(m: int, X: np.ndarray) -> np.ndarray:
    """psi W h^2 (Sec. 3.3, Eq. smoothint) with W from the derivative scheme."""
    h = np.pi / m
    return pou_weights(m) * geometry(m, X)["W"] * h * h


def area_volume(m: int, X: np.ndarray):
    """A = int 1, V = int (x, 0, 0) . n (Sec. 4.1 footnote), POU quadrature."""
    geo = geometry(m, X)
    w = pou_weights(m) * geo["W"] * (np.pi / m) ** 2
    return float(np.sum(w)), float(np.sum(w * X[:, 0] * geo["n"][:, 0]))
