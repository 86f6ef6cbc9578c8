"""Node numbering and physical coordinates (test infrastructure only).

Numbering (a reading; the paper fixes none): the volume node with GLL indices
(a0, a1[, a2]) is i = a0 + (p+1) a1 + (p+1)^2 a2. On the local face
f = 2*axis + side the face node j enumerates the tangential axes in increasing
axis order, first tangential axis fastest; the face node sits at a_axis = 0
(side 0) or a_axis = p (side 1). The map x = lo + h (r + 1) / 2 takes the
reference box [-1, 1]^d to the element (Sec. 2: axis-aligned quads/hexes).
"""
from __future__ import annotations

import numpy as np

from .basis import nodes_1d


def node_multi_index(dim, p):
    """[Np, dim] GLL index tuple of every volume node."""
    n1 = p + 1
    out = np.zeros((n1 ** dim, dim), dtype=np.int64)
    for i in range(n1 ** dim):
        rem = i
        for a in range(dim):
            out[i, a] = rem % n1
            rem //= n1
    return out


def face_volume_nodes(dim, p, f):
    """Volume node index of each face node on local face f, [Nfp]."""
    ax, side = divmod(f, 2)
    tang = [a for a in range(dim) if a != ax]
    n1 = p + 1
    nfp = n1 ** (dim - 1)
    out = np.zeros(nfp, dtype=np.int64)
    for j in range(nfp):
        idx = [0] * dim
        rem = j
        for t in tang:
            idx[t] = rem % n1
            rem //= n1
        idx[ax] = p if side else 0
        out[j] = sum(idx[a] * n1 ** a for a in range(dim))
    return out


def node_coords(mesh, p):
    """Physical coordinates of every volume node, [n_elem, Np, dim]."""
    dim = mesh["dim"]
    r, _ = nodes_1d(p)
    mi = node_multi_index(dim, p)
    ref = r[mi]  # [Np, dim]
    lo = mesh["elem_lo"][:, None, :]
    h = mesh["elem_h"][:, None, :]
    return lo + h * (ref[None, :, :] + 1.0) / 2.0


def face_point_coords(mesh, p, q):
    """Physical coordinates of the q^(d-1) Gauss points of every face,
    [n_face, Nqf, dim], from the minus element; tangential axes in increasing
    order, first tangential axis fastest."""
    from .basis import gauss
    dim = mesh["dim"]
    xi, _ = gauss(q)
    nqf = q ** (dim - 1)
    out = np.empty((mesh["n_face"], nqf, dim))
    for e in range(mesh["n_face"]):
        em = mesh["face_elem"][e, 0]
        ax, side = divmod(int(mesh["face_local"][e, 0]), 2)
        tang = [a for a in range(dim) if a != ax]
        lo, h = mesh["elem_lo"][em], mesh["elem_h"][em]
        for g in range(nqf):
            rem = g
            r = np.empty(dim)
            for t in tang:
                r[t] = xi[rem % q]
                rem //= q
            r[ax] = 1.0 if side else -1.0
            out[e, g] = lo + h * (r + 1.0) / 2.0
    return out


def face_node_coords(mesh, p):
    """Physical coordinates of every face node, [n_face, Nfp, dim], taken from
    the minus element."""
    x = node_coords(mesh, p)
    dim = mesh["dim"]
    out = np.empty((mesh["n_face"], (p + 1) ** (dim - 1), dim))
    for e in range(mesh["n_face"]):
        em = mesh["face_elem"][e, 0]
        fm = int(mesh["face_local"][e, 0])
        out[e] = x[em, face_volume_nodes(dim, p, fm)]
    return out
