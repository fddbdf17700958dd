"""Conforming correction of a nonconforming spectral element solution (oracle).

Test infrastructure only (see the package docstring).

Remark 4.3.0 and the proof of Lemma 3.3.1 (Appendix C.1): the nonconforming
solution u can be corrected into a conforming p in H^1 that vanishes on the
Dirichlet boundary and keeps an exponentially small H^1 error.  For elements of
the regular region with functions that are nonconforming on the wirebasket the
appendix makes three corrections, in this order:

1. delta: a trilinear function on the master cube with (u + delta)(n) = the
   average of u at every vertex n of the element over the elements that share
   it;
2. epsilon: for every edge S of the cube a function g along S, vanishing at
   its ends, blended by the bilinear factor of the other two variables
   ((1 -+ lambda_a) / 2 (1 -+ lambda_b) / 2), with (u + delta + epsilon)(t) =
   the average of u + delta at every point t of S;
3. nu: for every face the half jump of u + delta + epsilon across it, blended
   by the linear factor (1 -+ lambda) / 2 of the normal variable, so that both
   sides take the average on the face.

A last set of corrections makes p vanish on the Dirichlet boundary Gamma^[0]
(the appendix states it without formulas).  Reading: it is the same
construction with the target 0 instead of the average at every vertex, edge
point and face point of Gamma^[0] (the full trace instead of the half jump);
faces that are not Dirichlet faces (Neumann) are left free.

Every correction is of degree one in the blended variables and a trace
(degree W) in the others, so p lies in the same tensor-product space and is
computed here on the nodal values: box elements of workloads.MeshDesc (one
degree per problem; faces matching one to one, as the discretisation requires).
"""
from __future__ import annotations

import numpy as np

from .gll import gll


def _keys(mesh, e):
    """Rounded coordinates of the element's 8 corners (problem index first)."""
    lo, hi = mesh.elem_lo[e], mesh.elem_hi[e]
    pr = int(mesh.elem_problem[e])
    out = []
    for c in range(8):
        x = tuple(round(float(hi[a] if (c >> a) & 1 else lo[a]), 10) for a in range(3))
        out.append((pr,) + x)
    return out


def _dirichlet_faces(mesh):
    bc = getattr(mesh, "elem_bc", None)
    nbr = np.asarray(mesh.elem_nbr)
    dir_ = nbr == -1
    if bc is not None:
        dir_ = dir_ & (np.asarray(bc) == 0)
    return dir_


def conforming_correction(disc, U):
    """p = u + delta + epsilon + nu for a box-mesh Discretisation (one rhs)."""
    mesh = disc.mesh
    E = disc.E
    dirf = _dirichlet_faces(mesh)
    blocks = [disc.block(U, e).copy() for e in range(E)]   # [k][j][i], x fastest
    P = [disc.P[e] for e in range(E)]
    xs = [gll(P[e])[0] for e in range(E)]

    def lin(e, side):
        """(1 - x) / 2 or (1 + x) / 2 at the element's GLL nodes."""
        return (1.0 + xs[e]) / 2.0 if side else (1.0 - xs[e]) / 2.0

    def node_index(e, c):
        p = P[e] - 1
        return ((p if (c >> 2) & 1 else 0), (p if (c >> 1) & 1 else 0), (p if c & 1 else 0))

    # a vertex / edge / face point lies on Gamma^[0] if some element has a
    # Dirichlet face through it
    vkeys = [_keys(mesh, e) for e in range(E)]
    vert_members, vert_dir = {}, {}
    for e in range(E):
        for c in range(8):
            k = vkeys[e][c]
            vert_members.setdefault(k, []).append((e, c))
            on = any(dirf[e, 2 * a + ((c >> a) & 1)] for a in range(3))
            vert_dir[k] = vert_dir.get(k, False) or on

    # 1. delta (vertices): the targets from u itself
    vtarget = {k: 0.0 if vert_dir[k] else float(np.mean([blocks[m][node_index(m, cm)] for m, cm in mem]))
               for k, mem in vert_members.items()}
    for e in range(E):
        d = np.zeros(8)
        for c in range(8):
            d[c] = vtarget[vkeys[e][c]] - blocks[e][node_index(e, c)]
        corr = np.zeros_like(blocks[e])
        for c in range(8):
            fx, fy, fz = lin(e, c & 1), lin(e, (c >> 1) & 1), lin(e, (c >> 2) & 1)
            corr += d[c] * fz[:, None, None] * fy[None, :, None] * fx[None, None, :]
        blocks[e] = blocks[e] + corr

    # 2. epsilon (edges): edge along axis a with the other axes' sides (s1, s2)
    def edge_key(e, a, s):
        lo, hi = mesh.elem_lo[e], mesh.elem_hi[e]
        o = [b for b in range(3) if b != a]
        fixed = tuple(round(float(hi[b] if s[i] else lo[b]), 10) for i, b in enumerate(o))
        return (int(mesh.elem_problem[e]), a) + fixed + (round(float(lo[a]), 10), round(float(hi[a]), 10))

    def edge_trace(e, a, s, blk):
        o = [b for b in range(3) if b != a]
        p = P[e] - 1
        idx = [None, None, None]  # (i, j, k) = (x, y, z)
        for i, b in enumerate(o):
            idx[b] = p if s[i] else 0
        idx[a] = slice(None)
        return blk[idx[2], idx[1], idx[0]]

    edges = {}
    for e in range(E):
        for a in range(3):
            o = [b for b in range(3) if b != a]
            for s1 in (0, 1):
                for s2 in (0, 1):
                    k = edge_key(e, a, (s1, s2))
                    on = dirf[e, 2 * o[0] + s1] or dirf[e, 2 * o[1] + s2]
                    ent = edges.setdefault(k, [[], False])
                    ent[0].append((e, a, (s1, s2)))
                    ent[1] = ent[1] or on
    w = [b.copy() for b in blocks]
    for e in range(E):
        corr = np.zeros_like(blocks[e])
        for a in range(3):
            o = [b for b in range(3) if b != a]
            for s1 in (0, 1):
                for s2 in (0, 1):
                    members, on = edges[edge_key(e, a, (s1, s2))]
                    own = edge_trace(e, a, (s1, s2), w[e])
                    if on:
                        target = np.zeros_like(own)
                    else:
                        target = np.mean([edge_trace(m, am, sm, w[m]) for m, am, sm in members], axis=0)
                    g = target - own
                    f = [None, None, None]
                    f[a] = g
                    f[o[0]] = lin(e, s1)
                    f[o[1]] = lin(e, s2)
                    corr += f[2][:, None, None] * f[1][None, :, None] * f[0][None, None, :]
        blocks[e] = w[e] + corr

    # 3. nu (faces): face fi = 2 a + side, trace on the P x P face grid
    def face_trace(e, fi, blk):
        a, side = fi >> 1, fi & 1
        p = P[e] - 1
        n = p if side else 0
        if a == 0:
            return blk[:, :, n]
        if a == 1:
            return blk[:, n, :]
        return blk[n, :, :]

    v = [b.copy() for b in blocks]
    for e in range(E):
        corr = np.zeros_like(blocks[e])
        for fi in range(6):
            a, side = fi >> 1, fi & 1
            nb = int(mesh.elem_nbr[e, fi])
            own = face_trace(e, fi, v[e])
            if nb >= 0:
                target = 0.5 * (own + face_trace(nb, fi ^ 1, v[nb]))
            elif dirf[e, fi]:
                target = np.zeros_like(own)
            else:
                continue  # Neumann face: free
            c = target - own
            blend = lin(e, side)
            if a == 0:
                corr += c[:, :, None] * blend[None, None, :]
            elif a == 1:
                corr += c[:, None, :] * blend[None, :, None]
            else:
                corr += c[None, :, :] * blend[:, None, None]
        blocks[e] = v[e] + corr
    p = np.zeros(disc.ndof)
    for e in range(E):
        p[disc.off[e]:disc.off[e + 1]] = blocks[e].ravel()
    return p
