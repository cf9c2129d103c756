"""Host-side post-processing of macroscopic fields (NumPy): contact-angle and
Laplace-pressure measurement, drop height, saturation, information entropy.

These are measurements applied to outputs, not part of the time-stepping
method; they never touch the GPU and import neither the CUDA binding nor the
oracle.  Arrays are x-fastest: 2D fields have shape (ny, nx).
"""
import math

import numpy as np


def zero_contour_points(phi, mask=None):
    """Points where phi changes sign, by linear interpolation along rows and
    columns.  ``mask`` (same shape, bool) restricts to cells where it holds at
    both ends of the segment.  Returns an (n, 2) array of (x, y)."""
    pts = []
    ny, nx = phi.shape
    m = np.ones_like(phi, dtype=bool) if mask is None else mask
    a, b = phi[:, :-1], phi[:, 1:]
    ok = (a * b < 0) & m[:, :-1] & m[:, 1:]
    j, i = np.nonzero(ok)
    t = a[j, i] / (a[j, i] - b[j, i])
    pts.append(np.stack([i + t, j.astype(float)], 1))
    a, b = phi[:-1, :], phi[1:, :]
    ok = (a * b < 0) & m[:-1, :] & m[1:, :]
    j, i = np.nonzero(ok)
    t = a[j, i] / (a[j, i] - b[j, i])
    pts.append(np.stack([i.astype(float), j + t], 1))
    return np.concatenate(pts, 0)


def fit_circle(pts):
    """Algebraic (Kasa) least-squares circle fit; returns (xc, yc, R)."""
    x, y = pts[:, 0], pts[:, 1]
    A = np.stack([x, y, np.ones_like(x)], 1)
    b = x * x + y * y
    sol, *_ = np.linalg.lstsq(A, b, rcond=None)
    xc, yc = sol[0] / 2, sol[1] / 2
    R = math.sqrt(sol[2] + xc * xc + yc * yc)
    return xc, yc, R


def wall_level(phi0, x_col):
    """y of the phi0 = 1/2 level above the bottom wall along column ``x_col``
    (linear interpolation, first crossing from below)."""
    col = phi0[:, x_col]
    for j in range(len(col) - 1):
        if col[j] >= 0.5 > col[j + 1]:
            return j + (col[j] - 0.5) / (col[j] - col[j + 1])
    raise ValueError("no wall level found")


def contact_angle_flat(phi, phi0, D, margin=None):
    """Contact angle (degrees) of the phase-1 drop sitting on the bottom wall.

    The drop is the largest connected phase-1 region (phi > 0, outside the
    solid) that touches the wall layer; a circle is fitted to its phi = 0
    contour more than ``margin`` (default D) above the wall's phi0 = 1/2 level,
    and cos(theta) = (y_w - y_c)/R."""
    from scipy import ndimage

    ny, nx = phi.shape
    margin = D if margin is None else margin
    yw = wall_level(phi0, 0)
    fluid = phi0 < 1e-3
    liquid = (phi > 0) & (phi0 < 0.5)
    lab, n = ndimage.label(liquid, structure=np.ones((3, 3)))
    yy = np.arange(ny)[:, None] * np.ones((1, nx))
    near_wall = (yy >= yw) & (yy <= yw + D + 2)
    best, best_size = 0, 0
    for k in range(1, n + 1):
        comp = lab == k
        if not (comp & near_wall).any():
            continue
        size = int(comp.sum())
        if size > best_size:
            best, best_size = k, size
    if best == 0:
        raise ValueError("no drop attached to the wall")
    comp = lab == best
    # zero crossings on segments with one end inside the drop
    region = ndimage.binary_dilation(comp, structure=np.ones((3, 3))) & fluid
    mask = region & (yy > yw + margin)
    pts = zero_contour_points(phi, mask)
    xc, yc, R = fit_circle(pts)
    c = np.clip((yw - yc) / R, -1.0, 1.0)
    return math.degrees(math.acos(c)), dict(xc=xc, yc=yc, R=R, yw=yw, npts=len(pts))


def laplace_jump(P, centre, R, D, inner=2.0, outer=2.0):
    """Mean pressure inside r < R - inner*D minus mean outside r > R + outer*D
    (periodic minimum-image radius from ``centre`` = (x, y[, z]))."""
    shape = P.shape
    grids = np.meshgrid(*[np.arange(s, dtype=float) for s in shape], indexing="ij")
    X = list(reversed(grids))
    n = list(reversed(shape))
    r2 = np.zeros(shape)
    for a in range(len(shape)):
        d = X[a] - centre[a]
        d -= n[a] * np.floor(d / n[a] + 0.5)
        r2 += d * d
    r = np.sqrt(r2)
    return float(P[r < R - inner * D].mean() - P[r > R + outer * D].mean())


def drop_top_height(phi, x_centre, y_ref):
    """Height above ``y_ref`` of the phi = 0 crossing at the top of the drop in
    column ``x_centre`` (searching downward from the top of the box)."""
    col = phi[:, int(round(x_centre))]
    for j in range(len(col) - 1, 0, -1):
        if col[j] < 0 <= col[j - 1]:
            t = col[j - 1] / (col[j - 1] - col[j])
            return (j - 1 + t) - y_ref
    raise ValueError("no drop top found")


def saturation(phi, phi0):
    """Pore-volume fraction of phase 1: sum (1 - phi0)(1 + phi)/2 / sum (1 - phi0)."""
    w = 1.0 - phi0
    return float((w * 0.5 * (1.0 + phi)).sum() / w.sum())


def information_entropy(phi, bins=20, lo=-1.0, hi=1.0):
    """H(phi) = -sum p_n log2 p_n over ``bins`` equal value ranges of phi (Eq. 48)."""
    h, _ = np.histogram(np.clip(phi, lo, hi), bins=bins, range=(lo, hi))
    p = h / h.sum()
    p = p[p > 0]
    return float(-(p * np.log2(p)).sum())


def displacement_efficiency(phi, phi0, x_lo, x_hi):
    """De of Sec. 4.6: the share of fluid 1 (volume fraction (1 + phi)/2 of
    the fluid part 1 - phi0, phi0 the total solid indicator: walls and
    particles) found outside the cavity x_lo <= x <= x_hi."""
    fluid = np.clip(1.0 - phi0, 0.0, 1.0)
    # phase of the fluid part (phi is scaled by 1 - phi0 near solids)
    c = np.clip(phi / np.maximum(fluid, 1e-3), -1.0, 1.0)
    f1 = 0.5 * (1.0 + c) * fluid * (fluid > 0.01)
    x = np.arange(phi.shape[1])[None, :]
    out = (x < x_lo) | (x > x_hi)
    tot = f1.sum()
    return float((f1 * out).sum() / tot) if tot > 0 else 0.0


def interface_level(phi, x, y_lo, y_hi):
    """Height of the phi = 0 crossing (phase 1 below, phase 2 above) in column
    x between rows y_lo and y_hi, by linear interpolation; NaN if none."""
    col = np.asarray(phi)[y_lo:y_hi, x]
    idx = np.where((col[:-1] > 0) & (col[1:] <= 0))[0]
    if len(idx) == 0:
        return float("nan")
    i = idx[0]
    return float(y_lo + i + col[i] / (col[i] - col[i + 1]))
