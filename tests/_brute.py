"""Brute-force DARE reference for tiny grids (pure Python, FP64).

It pins the oracle's neighbourhood enumeration: instead of walking a window
around each pixel, it visits EVERY voxel of the grid and every sample in it,
and lets the distance kernel's own definition decide whether the voxel
contributes.  Orientation vectors come from quaternion products (v' = q v q*),
not from the rotation-matrix formula the oracle uses.
"""
import math

TENT, BOX, EXP = 0, 1, 2


def qmul(a, b):
    w1, x1, y1, z1 = a
    w2, x2, y2, z2 = b
    return (w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2,
            w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
            w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2,
            w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2)


def qrot(q, v):
    n = math.sqrt(sum(c * c for c in q))
    q = tuple(c / n for c in q)
    qc = (q[0], -q[1], -q[2], -q[3])
    r = qmul(qmul(q, (0.0, v[0], v[1], v[2])), qc)
    return r[1:]


def kernel_weight(kernel, R, g, c, k_dist):
    """Distance weight of voxel c for continuous voxel coordinate g, or None if c
    is outside the kernel's support."""
    d = [g[a] - c[a] for a in range(3)]
    if kernel == TENT:
        if any(abs(x) >= R for x in d):
            return None
        w = 1.0
        for x in d:
            w *= 1.0 - abs(x) / R
        return w
    if kernel == BOX:
        if any(abs(c[a] - math.floor(g[a] + 0.5)) > R for a in range(3)):
            return None
        return 1.0
    # EXP: support g - R < c <= g + R on every axis
    if any(not (-R < c[a] - g[a] <= R) for a in range(3)):
        return None
    return math.exp(-k_dist * math.sqrt(sum(x * x for x in d)) / R)


def reslice_pixel(dims, samples, g, plane_q, params):
    """samples: dict voxel (x, y, z) -> list of (value, quat).  params: oracle.Params."""
    ax_n = (0.0, 0.0, 1.0) if params.normal_axis == 1 else (0.0, 1.0, 0.0)
    n_r = qrot(plane_q, ax_n)
    x_r = qrot(plane_q, (1.0, 0.0, 0.0))
    cn = math.cos(math.radians(params.thr_normal_deg))
    ci = math.cos(math.radians(params.thr_inplane_deg))
    num = den = 0.0
    for cz in range(dims[2]):
        for cy in range(dims[1]):
            for cx in range(dims[0]):
                t = kernel_weight(params.kernel, params.radius, g, (cx, cy, cz), params.k_dist)
                if t is None:
                    continue
                for value, q in samples.get((cx, cy, cz), ()):
                    n_s = qrot(q, ax_n)
                    x_s = qrot(q, (1.0, 0.0, 0.0))
                    dn = sum(n_s[i] * n_r[i] for i in range(3))
                    di = abs(sum(x_s[i] * x_r[i] for i in range(3)))
                    if params.thr_normal_deg < 180 and dn < cn:
                        continue
                    if params.thr_inplane_deg < 180 and di < ci:
                        continue
                    w = math.exp(params.k_normal * (dn - 1) + params.k_inplane * (di - 1))
                    num += t * w * value
                    den += t * w
    if den > 0:
        return num / den, 1
    return params.unassigned, 0
