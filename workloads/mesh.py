"""Periodic box meshes of curvilinear hexahedra with rotated element frames.

Mesh format (identical to the C-ABI ``dg_mesh`` input):

* ``xgeo[e, c, k, j, i]``: physical coordinate ``c`` of element ``e`` sampled
  at the equispaced reference point ``(xi_i, xi_j, xi_k)``, ``xi_a = -1 + 2 a /
  ngeo``, in the element's own (local) frame; float64, ``i`` fastest.
* ``face_nbr[e, f] = (e2, f2, flip)``: local face ``f`` of element ``e`` touches
  local face ``f2`` of element ``e2``.  Local faces are numbered ``f = 2 d + s``
  with ``d`` the reference direction (0: xi, 1: eta, 2: zeta) and ``s = 0`` for
  the face at ``-1``, ``s = 1`` for the face at ``+1``.  A face node is indexed
  ``(p, q)`` along the two remaining reference directions in increasing order.
  ``flip`` (0..7) maps a face node ``(p, q)`` of ``(e, f)`` to the node
  ``(p2, q2)`` of ``(e2, f2)`` at the same physical point, for any polynomial
  degree ``N``: ``(a, b) = (q, p) if flip & 1 else (p, q)``;
  ``p2 = N - a if flip & 2 else a``; ``q2 = N - b if flip & 4 else b``.

Elements are the cells of a ``K^3`` lattice.  Each element's local frame is one
of the 24 proper rotations of the cube (seeded), so all relative face
orientations occur.  Geometry is sampled on an integer lattice so that points
shared by two elements are bitwise identical.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass

import numpy as np


def _proper_rotations():
    rots = []
    for perm in itertools.permutations(range(3)):
        for sg in itertools.product((1, -1), repeat=3):
            m = np.zeros((3, 3), dtype=np.int64)
            for a in range(3):
                m[perm[a], a] = sg[a]
            if round(np.linalg.det(m)) == 1:
                rots.append(m)
    return rots


# 24 signed permutation matrices with determinant +1.  Column a is the global
# direction of local axis a.
ROTATIONS = _proper_rotations()
assert len(ROTATIONS) == 24


def face_node_flip(flip: int, p, q, N: int):
    """Apply the ``flip`` code of the mesh format to face node (p, q)."""
    a, b = (q, p) if flip & 1 else (p, q)
    p2 = N - a if flip & 2 else a
    q2 = N - b if flip & 4 else b
    return p2, q2


def _sinpi(y):
    """sin(pi*y) with exact zeros at integer y (mesh deformation only)."""
    y = np.asarray(y, dtype=np.float64)
    r = y - 2.0 * np.round(y / 2.0)
    out = np.sin(np.pi * r)
    out[np.abs(r) == 1.0] = 0.0
    out[r == 0.0] = 0.0
    return out


@dataclass
class Mesh:
    K: int
    ngeo: int
    lo: float
    hi: float
    xgeo: np.ndarray          # [E, 3, ngeo+1, ngeo+1, ngeo+1] float64, i fastest
    face_nbr: np.ndarray      # [E, 6, 3] int32
    rot: np.ndarray           # [E] int, index into ROTATIONS

    @property
    def n_elems(self) -> int:
        return self.xgeo.shape[0]

    @property
    def volume(self) -> float:
        return (self.hi - self.lo) ** 3


def _local_lattice(R, ngeo):
    """Integer lattice offsets (within the element) of the local nodes.

    Returns [3, n, n, n] (global axis, k, j, i)."""
    n = ngeo + 1
    t = np.arange(n)
    loc = np.stack(np.meshgrid(t, t, t, indexing="ij")[::-1], 0)   # loc[a] = index along local axis a
    off = np.zeros((3, n, n, n), dtype=np.int64)
    for a in range(3):
        g = int(np.nonzero(R[:, a])[0][0])
        sg = int(R[g, a])
        off[g] += loc[a] if sg > 0 else ngeo - loc[a]
    return off


def box_mesh(K: int, ngeo: int, lo: float = -1.0, hi: float = 1.0,
             deform: str | None = None, amp: float = 0.1,
             rotate_seed: int | None = None, dims: tuple | None = None) -> Mesh:
    """Periodic ``K^3`` box mesh on ``[lo, hi]^3``.

    deform: None (Cartesian) or ``"sinprod"``: every coordinate is displaced by
    ``amp * prod_j sin(pi * y_j)`` with ``y`` the undeformed position scaled to
    ``[-1, 1]^3`` (zero on the box faces, so periodic faces still match).
    rotate_seed: None (identity frames) or the seed of each element's random
    proper rotation.
    dims: (Kx, Ky, Kz) elements per direction instead of K^3 (e.g. (2, 1, 1):
    two elements, each its own neighbour across its y and z faces).
    """
    Kd = tuple(int(k) for k in dims) if dims is not None else (K, K, K)
    if min(Kd) < 1 or ngeo < 1:
        raise ValueError("K and ngeo must be >= 1")
    E = Kd[0] * Kd[1] * Kd[2]
    n = ngeo + 1
    if rotate_seed is None:
        rot = np.zeros(E, dtype=np.int64)
        ident = next(i for i, m in enumerate(ROTATIONS) if (m == np.eye(3, dtype=np.int64)).all())
        rot[:] = ident
    else:
        rot = np.random.default_rng(rotate_seed).integers(0, 24, size=E)
    L = (np.array(Kd) * ngeo)[None, :, None, None, None]
    xgeo = np.empty((E, 3, n, n, n), dtype=np.float64)
    offs = [_local_lattice(R, ngeo) for R in ROTATIONS]
    eidx = np.arange(E)
    corner = np.stack([eidx % Kd[0], (eidx // Kd[0]) % Kd[1], eidx // (Kd[0] * Kd[1])], 1) * ngeo
    for r in np.unique(rot):
        sel = np.nonzero(rot == r)[0]
        lat = offs[r][None] + corner[sel][:, :, None, None, None]
        y = lo + (hi - lo) * (lat / L)
        if deform == "sinprod":
            s = -1.0 + 2.0 * lat / L
            dsp = amp * _sinpi(s[:, 0]) * _sinpi(s[:, 1]) * _sinpi(s[:, 2]) * (hi - lo) / 2.0
            y = y + dsp[:, None]
        elif deform is not None:
            raise ValueError(deform)
        xgeo[sel] = y
    face_nbr = _connectivity(Kd, rot)
    return Mesh(K=Kd[0], ngeo=ngeo, lo=lo, hi=hi, xgeo=xgeo, face_nbr=face_nbr, rot=rot)


def _face_lattice_points(R, d, s, ec, t):
    """Global lattice points (unwrapped) of a local face's nodes at a lattice
    resolution where the element spans [0, t]; returns [n, n, 3] indexed (p, q)."""
    n = t + 1
    pts = np.zeros((n, n, 3), dtype=np.int64)
    tang = [a for a in range(3) if a != d]
    for p in range(n):
        for q in range(n):
            loc = [0, 0, 0]
            loc[d] = s * t
            loc[tang[0]] = p
            loc[tang[1]] = q
            g = np.array(ec) * t
            for a in range(3):
                ga = int(np.nonzero(R[:, a])[0][0])
                sg = int(R[ga, a])
                g[ga] += loc[a] if sg > 0 else t - loc[a]
            pts[p, q] = g
    return pts


def _orientation_table():
    """(f2, flip) for every (rotation of e, local face f, rotation of e2):
    the relative orientation does not depend on the element positions."""
    tab = np.zeros((24, 6, 24, 2), dtype=np.int64)
    t = 2
    ec = (1, 1, 1)
    for r1, R in enumerate(ROTATIONS):
        for f in range(6):
            d, s = divmod(f, 2)
            gax = int(np.nonzero(R[:, d])[0][0])
            gsg = int(R[gax, d]) * (2 * s - 1)
            ec2 = list(ec)
            ec2[gax] += gsg
            P1 = _face_lattice_points(R, d, s, ec, t)
            for r2, R2 in enumerate(ROTATIONS):
                d2 = int(np.nonzero(R2[gax, :])[0][0])
                s2 = 1 if int(R2[gax, d2]) * (-gsg) > 0 else 0
                P2 = _face_lattice_points(R2, d2, s2, ec2, t)
                found = -1
                for flip in range(8):
                    if all((P1[p, q] == P2[face_node_flip(flip, p, q, t)]).all()
                           for p in range(t + 1) for q in range(t + 1)):
                        found = flip
                        break
                if found < 0:
                    raise RuntimeError("no face orientation found")
                tab[r1, f, r2] = (2 * d2 + s2, found)
    return tab


_ORIENT = None


def _connectivity(Kd, rot: np.ndarray) -> np.ndarray:
    global _ORIENT
    if _ORIENT is None:
        _ORIENT = _orientation_table()
    Kd = np.array(Kd)
    E = int(Kd.prod())
    e = np.arange(E)
    ec = np.stack([e % Kd[0], (e // Kd[0]) % Kd[1], e // (Kd[0] * Kd[1])], 1)
    nbr = np.zeros((E, 6, 3), dtype=np.int32)
    Rs = np.stack(ROTATIONS)                      # [24, 3, 3]
    for f in range(6):
        d, s = divmod(f, 2)
        col = Rs[rot][:, :, d]                    # [E, 3] global image of local axis d
        gax = np.argmax(np.abs(col), axis=1)
        gsg = col[np.arange(E), gax] * (2 * s - 1)
        ec2 = ec.copy()
        ec2[np.arange(E), gax] = (ec2[np.arange(E), gax] + gsg) % Kd[gax]
        e2 = ec2[:, 0] + Kd[0] * (ec2[:, 1] + Kd[1] * ec2[:, 2])
        ft = _ORIENT[rot, f, rot[e2]]
        nbr[:, f, 0] = e2
        nbr[:, f, 1] = ft[:, 0]
        nbr[:, f, 2] = ft[:, 1]
    return nbr


# ---------------------------------------------------------------------------
# Non-conforming meshes: a periodic K^3 box whose selected cells are split into
# 2 x 2 x 2 children.  A face between an unsplit cell and a split neighbour is
# a mortar: the big face meets four small faces.
#
# Additional format (identical to the C-ABI ``dg_mesh`` mortar fields):
# * ``mortars[m] = (eB, fB, eS0, fS0, flip0, ..., eS3, fS3, flip3)``: the big
#   face ``fB`` of element ``eB`` is split into quadrants k = a + 2 b, (a, b)
#   the halves along its face-local (p, q) directions; quadrant k is local
#   face ``fS_k`` of element ``eS_k``, and ``flip_k`` maps a node (p, q) of the
#   quadrant, numbered in the big face's directions, to the small face's own
#   node (the ``flip`` code of the conforming faces).
# * ``face_nbr[e, f] = (-1 - m, 0, 0)`` on the big side of mortar m and
#   ``(-1 - m, k, 0)`` on its quadrant k.
@dataclass
class MortarMesh(Mesh):
    mortars: np.ndarray = None   # [M, 14] int32
    size: np.ndarray = None      # [E] element edge in fine lattice units (2: unsplit, 1: child)
    origin: np.ndarray = None    # [E, 3] lower corner in fine lattice units


def refined_box_mesh(K: int, refine, lo: float = -1.0, hi: float = 1.0, rotate_seed: int | None = None) -> MortarMesh:
    """Periodic Cartesian ``K^3`` box (ngeo = 1) with the cells where
    ``refine`` (a boolean array of K^3 entries, cell index x fastest) is true
    split into eight children.  Elements: the cells in order, a split cell
    replaced by its eight children (x fastest).  Element frames are seeded
    proper rotations (identity if rotate_seed is None); all connectivity,
    mortar quadrants and flips are found by matching corner points."""
    refine = np.asarray(refine, dtype=bool).reshape(-1)
    if refine.size != K ** 3:
        raise ValueError("refine needs K^3 entries")
    L = 2 * K                                     # the periodic box in fine lattice units
    origin, size = [], []
    for cell in range(K ** 3):
        c = np.array([cell % K, (cell // K) % K, cell // (K * K)]) * 2
        if refine[cell]:
            for ch in range(8):
                origin.append(c + np.array([ch & 1, (ch >> 1) & 1, (ch >> 2) & 1]))
                size.append(1)
        else:
            origin.append(c)
            size.append(2)
    origin = np.array(origin, dtype=np.int64)
    size = np.array(size, dtype=np.int64)
    E = len(size)
    if rotate_seed is None:
        ident = next(i for i, m in enumerate(ROTATIONS) if (m == np.eye(3, dtype=np.int64)).all())
        rot = np.full(E, ident, dtype=np.int64)
    else:
        rot = np.random.default_rng(rotate_seed).integers(0, 24, size=E)
    # corner lattice points of each element's local reference cube [E][8][3] (local corner index i + 2 j + 4 k)
    xgeo = np.empty((E, 3, 2, 2, 2), dtype=np.float64)
    corners = np.empty((E, 2, 2, 2, 3), dtype=np.int64)
    for e in range(E):
        R = ROTATIONS[rot[e]]
        off = _local_lattice(R, 1)                # [3, k, j, i] in {0, 1}
        pts = origin[e][:, None, None, None] + size[e] * off
        corners[e] = np.moveaxis(pts, 0, -1)
        xgeo[e] = lo + (hi - lo) * pts / L
    # face corner points, face-local (p, q) order, wrapped into the box
    def face_pts(e, f):
        d, s = divmod(f, 2)
        tang = [a for a in range(3) if a != d]
        out = np.empty((2, 2, 3), dtype=np.int64)
        for p in range(2):
            for q in range(2):
                loc = [0, 0, 0]
                loc[d] = s
                loc[tang[0]] = p
                loc[tang[1]] = q
                out[p, q] = corners[e, loc[2], loc[1], loc[0]]
        return out
    # a face is identified by its centre (four times it, wrapped into the box):
    # corner sets alone are ambiguous in a box two cells wide
    key = lambda pts: tuple(int(v) % (4 * L) for v in pts.reshape(-1, 3).sum(0))
    index = {}
    for e in range(E):
        for f in range(6):
            index.setdefault(key(face_pts(e, f)), []).append((e, f))

    def flip_between(P1, P2):
        for flip in range(8):
            if all(((P1[p, q] - P2[face_node_flip(flip, p, q, 1)]) % L == 0).all() for p in range(2) for q in range(2)):
                return flip
        raise RuntimeError("no face orientation found")

    face_nbr = np.zeros((E, 6, 3), dtype=np.int32)
    done = np.zeros((E, 6), dtype=bool)
    mortars = []
    for e in range(E):
        for f in range(6):
            if done[e, f]:
                continue
            P1 = face_pts(e, f)
            others = [x for x in index[key(P1)] if x != (e, f)]
            if others:                            # conforming (same size on both sides)
                (e2, f2), = others
                face_nbr[e, f] = (e2, f2, flip_between(P1, face_pts(e2, f2)))
                face_nbr[e2, f2] = (e, f, flip_between(face_pts(e2, f2), P1))
                done[e, f] = done[e2, f2] = True
                continue
            if size[e] != 2:
                continue                          # a small face: registered from its big side
            m = len(mortars)
            rec = [e, f]
            for k in range(4):
                a, b = k & 1, k >> 1
                Q = np.empty((2, 2, 3), dtype=np.int64)
                for p in range(2):
                    for q in range(2):
                        Q[p, q] = P1[0, 0] + ((a + p) * (P1[1, 0] - P1[0, 0]) + (b + q) * (P1[0, 1] - P1[0, 0])) // 2
                cand = index.get(key(Q), [])
                if len(cand) != 1:
                    raise RuntimeError("mortar quadrant not matched")
                (es, fs), = cand
                rec += [es, fs, flip_between(Q, face_pts(es, fs))]
                face_nbr[es, fs] = (-1 - m, k, 0)
                done[es, fs] = True
            face_nbr[e, f] = (-1 - m, 0, 0)
            done[e, f] = True
            mortars.append(rec)
    if not done.all():
        raise RuntimeError("unmatched faces: a split cell next to an unsplit one needs 2:1 balance")
    return MortarMesh(K=K, ngeo=1, lo=lo, hi=hi, xgeo=xgeo, face_nbr=face_nbr, rot=rot,
                      mortars=np.array(mortars, dtype=np.int32).reshape(-1, 14), size=size, origin=origin)
