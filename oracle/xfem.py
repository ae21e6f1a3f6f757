"""FP64 CPU oracle of the X-FFT solver for periodic 3D linear-elastic homogenization.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  Every routine restates the method of
arXiv 2601.02172 in plain NumPy/SciPy, following the paper's order and notation:

* the X-FEM space with modified abs enrichment (Sec. 2.1, eqs. X-FEM_space, enrichedN,
  levelset, modifiedabsEnrichment) on voxels split into six P1 tetrahedra (Sec. 3, Fig. P16);
* the internal scaling of the enriched functions (Sec. 2.2, eqs. scaledEnrichedFunction,
  XFFT_diagonal, L2X), read per degree of freedom;
* the element matrices and vectors by sub-tetrahedron quadrature with the 4-point degree-2
  rule (Sec. 3, eqs. Kapp, b, Kapp_q, b_q, Sapp_q) after splitting each cut P1 element along
  the linearised interface (snap threshold for nodal level-set values, Sec. 3);
* global assembly (eq. linearSystem_element), the X-FFT block preconditioner
  ``P = diag(A0_11, I)`` (eqs. scaledPreconditioner, constantCoefficientPreconditioner), the
  Fourier symbol of ``A0_11`` built from the voxel matrix (eqs. A0Voxel, GreenHermitian), the
  linear CG of Algorithm 1 with the stopping rule of eqs. stoppingCriterion/convergence;
* average stress, effective stiffness (stress form and energy form, App. A identity) and the
  derivative of the effective stiffness with respect to the phase Lame constants and a
  per-voxel modulus scale (envelope identity of App. A; not in the paper's experiments).

Readings of silent or garbled passages (Kuhn split, sign of the residual, per-DOF scaling,
snap units, cell-volume normalisation of the stopping rule, ...) are stated where they are used.

Parity pins (tests/test_oracle_*.py): homogeneous cells, the tilted laminate's closed form,
Voigt/Reuss bounds, symmetry, axis-permutation invariance, PCG = direct solve, dense
brute-force eigen-analysis on tiny grids, FFT symbol = assembled operator, quadrature
exactness, sub-tetrahedron volumes, the DOF overhead printed for Hashin's inclusion, finite
differences and Euler homogeneity of the gradient; with several interfaces (Sec. 4.2's coated
sphere) the three-layer laminate's closed form, Hashin's neutral-inclusion bulk modulus and the
reduction to one interface.
"""
from __future__ import annotations

import itertools
import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

SQ2 = math.sqrt(2.0)
# Voigt-Mandel component order (11, 22, 33, 23, 13, 12), shear entries carry sqrt(2).
MANDEL_PAIRS = ((0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1))
# Six P1 tetrahedra per voxel: one per permutation (p, q, r) of the axes, with vertices
# o, o+e_p, o+e_p+e_q, o+(1,1,1) (the split around the main voxel diagonal).
KUHN_PERMS = tuple(itertools.permutations(range(3)))
# Node numbering of the voxel corners, matrix Y of Sec. 3 (before eq. GreenHermitian).
VOXEL_CORNERS = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0],
                          [0, 0, 1], [1, 0, 1], [1, 1, 1], [0, 1, 1]], dtype=np.int64)


def mandel_extraction():
    """Matrix M (6x9) that maps a displacement gradient H (row-major, H[i,j] = du_i/dx_j) to
    the Mandel vector of its symmetric part (eq. shapeFunctionGradient)."""
    M = np.zeros((6, 9))
    for r, (i, j) in enumerate(MANDEL_PAIRS):
        if i == j:
            M[r, 3 * i + j] = 1.0
        else:
            M[r, 3 * i + j] = SQ2 / 2.0
            M[r, 3 * j + i] = SQ2 / 2.0
    return M


_M = mandel_extraction()


def iso_stiffness(lam, mu):
    """Isotropic stiffness lam I(x)I + 2 mu I_sym as a 6x6 Mandel matrix."""
    m = np.array([1.0, 1.0, 1.0, 0.0, 0.0, 0.0])
    return lam * np.outer(m, m) + 2.0 * mu * np.eye(6)


def symgrad_operator(grads):
    """Symmetric-gradient operator B = M (grad N (x) I_3) of eq. shapeFunctionGradient.

    ``grads`` has shape (..., nf, 3) (scalar gradients of nf shape functions).  Returns
    (..., 6, 3 nf) with column ``3 a + c`` the Mandel strain of ``N_a e_c``.
    """
    grads = np.asarray(grads, dtype=float)
    nf = grads.shape[-2]
    lead = grads.shape[:-2]
    H = np.zeros(lead + (nf, 3, 3, 3))  # [a, c, i, j]: du_i/dx_j for N_a e_c
    for c in range(3):
        H[..., :, c, c, :] = grads
    Hf = H.reshape(lead + (nf, 3, 9))
    B = np.einsum("rk,...ack->...rac", _M, Hf)
    return B.reshape(lead + (6, 3 * nf))


def quad4():
    """Symmetric 4-point rule on the reference tetrahedron, exact for quadratics.

    Barycentric points are the permutations of (a, b, b, b) with a = (5 + 3 sqrt5)/20 and
    b = (5 - sqrt5)/20, equal weights 1/4 (times the volume); the paper's 4-point rule of
    Shunn and Ham integrates the same quadratic integrands exactly (Sec. 3).
    """
    a = (5.0 + 3.0 * math.sqrt(5.0)) / 20.0
    b = (5.0 - math.sqrt(5.0)) / 20.0
    bary = np.full((4, 4), b)
    np.fill_diagonal(bary, a)
    return bary, np.full(4, 0.25)


_QB, _QW = quad4()


def tet_volume(P):
    P = np.asarray(P, dtype=float)
    return abs(float(np.linalg.det(np.stack([P[1] - P[0], P[2] - P[0], P[3] - P[0]])))) / 6.0


def clip_tet(X, L, s):
    """Sub-tetrahedra covering {x in T : s * L_h(x) >= 0} for the P1 interpolant L_h.

    Generic convex clip (independent of any case table): each face of T is clipped against the
    half-space, the interface polygon {L_h = 0} is added as one more face, and every boundary
    triangle is joined to an interior apex.  Returns a list of 4x3 vertex arrays.  This is
    the subdivision of Sec. 3 (Fig. subdivision) up to how the convex pieces are cut into
    tetrahedra, which does not change any integral.
    """
    X = np.asarray(X, dtype=float)
    L = np.asarray(L, dtype=float)
    inside = s * L >= 0.0

    def cross(i, j):
        t = L[i] / (L[i] - L[j])
        return X[i] + t * (X[j] - X[i])

    faces = ((0, 1, 2), (0, 1, 3), (0, 2, 3), (1, 2, 3))
    polys = []
    for f in faces:
        poly = []
        for m in range(3):
            i, j = f[m], f[(m + 1) % 3]
            if inside[i]:
                poly.append(X[i])
            if L[i] * L[j] < 0.0:
                poly.append(cross(i, j))
        if len(poly) >= 3:
            polys.append(poly)
    cut = [X[i] for i in range(4) if L[i] == 0.0]
    for i in range(4):
        for j in range(i + 1, 4):
            if L[i] * L[j] < 0.0:
                cut.append(cross(i, j))
    if len(cut) >= 3:
        C = np.array(cut)
        ctr = C.mean(axis=0)
        # plane normal: gradient of L_h
        J = np.stack([X[1] - X[0], X[2] - X[0], X[3] - X[0]])
        g = np.linalg.solve(J, L[1:] - L[0])
        nrm = g / np.linalg.norm(g)
        u = C[0] - ctr
        u = u - nrm * (u @ nrm)
        if np.linalg.norm(u) == 0.0:
            u = C[1] - ctr
            u = u - nrm * (u @ nrm)
        u /= np.linalg.norm(u)
        v = np.cross(nrm, u)
        ang = np.arctan2((C - ctr) @ v, (C - ctr) @ u)
        polys.append([C[k] for k in np.argsort(ang)])
    verts = [X[i] for i in range(4) if inside[i]]
    for i in range(4):
        for j in range(i + 1, 4):
            if L[i] * L[j] < 0.0:
                verts.append(cross(i, j))
    apex = np.mean(np.array(verts), axis=0)
    out = []
    for poly in polys:
        for m in range(1, len(poly) - 1):
            out.append(np.array([apex, poly[0], poly[m], poly[m + 1]]))
    return out


def classify(L, n, tau):
    """Cut flags (nvox, 6) and enriched node set of a nodal level set (Sec. 2.1 and Sec. 3):
    after snapping |L| < tau to 0, a tet is cut iff its vertex values take both signs, and
    the enriched nodes are all nodes of cut tets."""
    n = tuple(int(v) for v in n)
    Ls = np.where(np.abs(L) < tau, 0.0, np.asarray(L, float)).ravel()
    i, j, k = np.meshgrid(np.arange(n[0]), np.arange(n[1]), np.arange(n[2]), indexing="ij")
    ijk = np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1)
    cut = np.zeros((ijk.shape[0], 6), bool)
    nodes_all = []
    for t, (p, q, r) in enumerate(KUHN_PERMS):
        off = np.zeros((4, 3), dtype=np.int64)
        off[1, p] = 1
        off[2, p] = 1
        off[2, q] = 1
        off[3, :] = 1
        idx = np.stack([((ijk + off[a]) % n) @ np.array([n[1] * n[2], n[2], 1]) for a in range(4)], 1)
        Lt = Ls[idx]
        cut[:, t] = (Lt.min(1) < 0) & (Lt.max(1) > 0)
        nodes_all.append(idx[cut[:, t]])
    return cut, np.unique(np.concatenate(nodes_all).ravel())


class XFEM:
    """The discrete X-FFT cell problem of one microstructure.

    Parameters
    ----------
    L : nodal level set, shape ``n`` (C order), ``L < 0`` = phase "minus"; or, with
        ``phases``, K nodal level sets, shape ``(K,) + n``.
    n : voxels per axis (N1, N2, N3); length: cell edge lengths.
    lame_minus, lame_plus : (lambda, mu) of the ``L < 0`` and ``L > 0`` phases.
    phases : several interfaces (Sec. 4.2's coated sphere): K + 1 pairs (lambda, mu).  A point
        belongs to phase k, the index of the first level set that is negative there, or to
        phase K where none is.  Each interface k is the zero set of L_k where the level sets
        before it are positive; a cut tet is cut by one interface only (the paper's setting:
        one interface per element) and is enriched with the modified abs of that interface's
        level set.  The enrichment function of a node is then the sum of the per-interface
        functions, which have disjoint supports.  One level set with (lame_minus, lame_plus)
        is the case K = 1.
    scale : optional per-voxel modulus scale s_v (shape ``n``); C = s_v C_phase.
    tau : snap threshold; nodal values with |L| < tau become 0 (Sec. 3: "below 1e-6").
          Default ``1e-6 * min(h)`` (the paper's absolute 1e-6 at its N = 16, h ~ 1 um scale).

    DOF numbering (shared with nothing; chosen to make comparisons easy): standard DOF
    (node n, component c) -> ``c * nFE + n``; scaled enriched DOF (enriched id j, component
    c) -> ``3 nFE + c * nX + j``; enriched ids follow increasing node index.
    """

    def __init__(self, L, n, length=(1.0, 1.0, 1.0), lame_minus=(1.0, 1.0),
                 lame_plus=(1.0, 1.0), scale=None, tau=None, phases=None, enrichment=True):
        self.n = tuple(int(v) for v in n)
        self.length = tuple(float(v) for v in length)
        self.h = np.array([self.length[a] / self.n[a] for a in range(3)])
        self.nFE = int(np.prod(self.n))
        self.nvox = self.nFE
        self.volY = float(np.prod(self.length))
        self.tau = 1e-6 * float(np.min(self.h)) if tau is None else float(tau)
        if phases is None:
            phases = (lame_minus, lame_plus)
            L = np.asarray(L, dtype=float).reshape((1,) + self.n)
        else:
            L = np.asarray(L, dtype=float).reshape((-1,) + self.n)
        self.nL = L.shape[0]
        if len(phases) != self.nL + 1:
            raise ValueError("K level sets need K + 1 phases")
        self.Ls = np.where(np.abs(L) < self.tau, 0.0, L).reshape(self.nL, -1)
        self.L = self.Ls[0]
        self.phases = [tuple(map(float, p)) for p in phases]
        self.scale = (np.ones(self.nvox) if scale is None
                      else np.asarray(scale, dtype=np.float64).ravel().copy())
        self.enrichment = bool(enrichment)
        self._geometry()
        self._classify()
        self._cut_quadrature()
        self.ndof = 3 * (self.nFE + self.nX)

    # ------------------------------------------------------------------ geometry
    def node_index(self, ijk):
        ijk = np.asarray(ijk) % np.asarray(self.n)
        return (ijk[..., 0] * self.n[1] + ijk[..., 1]) * self.n[2] + ijk[..., 2]

    def _geometry(self):
        n = self.n
        i, j, k = np.meshgrid(np.arange(n[0]), np.arange(n[1]), np.arange(n[2]), indexing="ij")
        self.vox_ijk = np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1)
        self.tet_offsets = []
        self.tet_grads = []
        self.tet_vol = []
        nodes = np.zeros((self.nvox, 6, 4), dtype=np.int64)
        for t, (p, q, r) in enumerate(KUHN_PERMS):
            off = np.zeros((4, 3), dtype=np.int64)
            off[1, p] = 1
            off[2, p] = 1
            off[2, q] = 1
            off[3, :] = 1
            self.tet_offsets.append(off)
            X = off * self.h
            J = np.stack([X[1] - X[0], X[2] - X[0], X[3] - X[0]])  # rows: edge vectors
            Jinv = np.linalg.inv(J)
            # barycentric N_b (b = 1..3) = (Jinv^T (x - X0))_b ; grad N_b = column b of Jinv
            G = np.zeros((4, 3))
            G[1:] = Jinv.T
            G[0] = -G[1:].sum(axis=0)
            self.tet_grads.append(G)
            self.tet_vol.append(abs(np.linalg.det(J)) / 6.0)
            for a in range(4):
                nodes[:, t, a] = self.node_index(self.vox_ijk + off[a])
        self.tet_nodes = nodes
        self.B_std = [symgrad_operator(G) for G in self.tet_grads]  # 6 x 12 per tet type

    def _classify(self):
        if not self.enrichment:
            return self._classify_p1()
        K = self.nL
        Lt = self.Ls[:, self.tet_nodes]  # (K, nvox, 6, 4)
        neg = Lt.min(axis=3) < 0.0
        pos = Lt.max(axis=3) > 0.0
        # first level set negative somewhere on the tet (K if none): the phase of an uncut tet
        # (a tet whose vertices are all 0 lies on the interface; it gets the plus phase), the
        # minus phase of a cut one
        first = np.where(neg.any(axis=0), neg.argmax(axis=0), K)
        kk = np.minimum(first, K - 1)
        self.cut = (first < K) & np.take_along_axis(pos, kk[None], axis=0)[0]
        self.tet_phase = first
        J = np.unique(self.tet_nodes[self.cut])
        self.enr_nodes = J
        self.nX = int(J.size)
        self.enr_id = -np.ones(self.nFE, dtype=np.int64)
        self.enr_id[J] = np.arange(self.nX)
        cv, ct = np.nonzero(self.cut)
        self.cut_list = np.stack([cv, ct], axis=1) if cv.size else np.zeros((0, 2), np.int64)
        # interface of each cut tet and the phases of its minus and plus sides: the plus side
        # lies in the first later level set that is negative on the tet, else in phase K; a
        # later level set that also changes sign there would put two interfaces in one element
        ki = first[cv, ct]
        later = np.arange(K)[:, None] > ki[None, :]
        lneg = neg[:, cv, ct] & later
        if np.any(lneg & pos[:, cv, ct]):
            raise ValueError("a tet is cut by two interfaces")
        pp = np.where(lneg.any(axis=0), lneg.argmax(axis=0), K)
        self.cut_iface = ki
        self.cut_phase = {-1: ki, +1: pp}

    def _classify_p1(self):
        """The P1 baseline of the discretization table (Sec. 4.1): voxel-segmented P1 elements
        without enrichment.  Each voxel takes one phase, that of its centre, where the level set
        is the trilinear interpolant of the corner values, i.e. their mean; with several level
        sets the first one negative at the centre decides (phase K if none is).  Nothing is cut
        and nothing is enriched."""
        K = self.nL
        corners = self.node_index(self.vox_ijk[:, None, :] + VOXEL_CORNERS[None, :, :])  # (nvox, 8)
        centre = self.Ls[:, corners].mean(axis=2)  # (K, nvox)
        neg = centre < 0.0
        first = np.where(neg.any(axis=0), neg.argmax(axis=0), K)
        self.tet_phase = np.repeat(first[:, None], 6, axis=1)
        self.cut = np.zeros((self.nvox, 6), bool)
        self.enr_nodes = np.zeros(0, dtype=np.int64)
        self.nX = 0
        self.enr_id = -np.ones(self.nFE, dtype=np.int64)
        self.cut_list = np.zeros((0, 2), np.int64)
        self.cut_iface = np.zeros(0, dtype=np.int64)
        self.cut_phase = {-1: np.zeros(0, dtype=np.int64), +1: np.zeros(0, dtype=np.int64)}

    # ------------------------------------------------------------------ cut elements
    def _cut_tet_points(self, v, t, k):
        """Quadrature data of cut tet (v, t) of interface k: per side, points' barycentric
        coordinates and weights, for the sub-tetrahedra of the linearised interface (Sec. 3)."""
        off = self.tet_offsets[t]
        X = off * self.h
        Lv = self.Ls[k][self.tet_nodes[v, t]]
        J = np.stack([X[1] - X[0], X[2] - X[0], X[3] - X[0]])
        Jinv = np.linalg.inv(J)
        sides = {}
        for s in (+1, -1):
            bary, wts = [], []
            for P in clip_tet(X, Lv, s):
                vol = tet_volume(P)
                pts = _QB @ P  # (4, 3)
                lam = (pts - X[0]) @ Jinv  # barycentric 1..3
                b = np.concatenate([1.0 - lam.sum(axis=1, keepdims=True), lam], axis=1)
                bary.append(b)
                wts.append(_QW * vol)
            sides[s] = (np.concatenate(bary), np.concatenate(wts))
        return Lv, sides

    def _enriched_B(self, G, Lv, s, bary):
        """Unscaled symmetric gradients of the 4 enriched functions N_a rho^m on side s.

        On side s the modified abs enrichment is rho = sum_b N_b (|L_b| - s L_b)
        (eq. modifiedabsEnrichment with |L_h| = s L_h), so grad(N_a rho) =
        rho grad N_a + N_a grad rho (eq. enrichedN).  Returns (nq, 6, 12).
        """
        coef = np.abs(Lv) - s * Lv
        rho = bary @ coef  # (nq,)
        grho = G.T @ coef  # (3,)
        gX = rho[:, None, None] * G[None, :, :] + bary[:, :, None] * grho[None, None, :]
        return symgrad_operator(gX)

    def _cut_quadrature(self):
        """Scaling factors D0 per enriched DOF (eq. XFFT_diagonal, per-DOF reading) and the
        quadrature data of every cut tet."""
        self.D = np.zeros((self.nX, 3))
        # Dblk[j] = int sym(grad N_X^j (x) e_k) : sym(grad N_X^j (x) e_l), k, l = 1..3: the 3x3
        # node block of the enriched-enriched reference Gram matrix; its diagonal is D0
        self.Dblk = np.zeros((self.nX, 3, 3))
        self.cut_data = []
        for (v, t), k in zip(self.cut_list, self.cut_iface):
            Lv, sides = self._cut_tet_points(v, t, k)
            G = self.tet_grads[t]
            eids = self.enr_id[self.tet_nodes[v, t]]
            for s in (+1, -1):
                bary, w = sides[s]
                BX = self._enriched_B(G, Lv, s, bary)  # (nq, 6, 12)
                sq = np.einsum("q,qrk->k", w, BX * BX).reshape(4, 3)
                gram = np.einsum("q,qrk,qrl->kl", w, BX, BX)  # (12, 12)
                for a in range(4):
                    self.D[eids[a]] += sq[a]
                    self.Dblk[eids[a]] += gram[3 * a:3 * a + 3, 3 * a:3 * a + 3]
            self.cut_data.append((Lv, sides))
        if self.nX and np.any(self.D <= 0.0):
            raise ValueError("non-positive enrichment scaling factor")
        self.Dinvsqrt = 1.0 / np.sqrt(self.D) if self.nX else np.zeros((0, 3))
        # scaled blocks (unit diagonal): the variant enriched preconditioner's 3x3 blocks
        self.Bblk = self.Dblk * self.Dinvsqrt[:, :, None] * self.Dinvsqrt[:, None, :]

    def _C(self, p, v):
        """Stiffness of phase p in voxel v."""
        lam, mu = self.phases[p]
        return self.scale[v] * iso_stiffness(lam, mu)

    def _side_phase(self, idx, s):
        return int(self.cut_phase[s][idx])

    def cut_element(self, idx):
        """Scaled element matrix (24x24), stress matrix (6x24, eq. Sapp_q) and DOF indices of
        the idx-th cut tet; local DOF order: std (3a+c), then enriched (12 + 3a + c)."""
        v, t = self.cut_list[idx]
        Lv, sides = self.cut_data[idx]
        G = self.tet_grads[t]
        nodes = self.tet_nodes[v, t]
        eids = self.enr_id[nodes]
        scale = np.concatenate([np.ones(12), self.Dinvsqrt[eids].ravel()])
        K = np.zeros((24, 24))
        S = np.zeros((6, 24))
        Bs = self.B_std[t]
        for s in (+1, -1):
            bary, w = sides[s]
            BX = self._enriched_B(G, Lv, s, bary)
            Bf = np.concatenate([np.broadcast_to(Bs, BX.shape), BX], axis=2) * scale
            C = self._C(self._side_phase(idx, s), v)
            CB = np.matmul(C, Bf)  # (nq, 6, 24)
            K += np.tensordot(Bf * w[:, None, None], CB, axes=([0, 1], [0, 1]))
            S += np.tensordot(w, CB, axes=(0, 0))
        dofs = np.concatenate([
            (np.arange(3)[None, :] * self.nFE + nodes[:, None]).ravel(),
            (3 * self.nFE + np.arange(3)[None, :] * self.nX + eids[:, None]).ravel()])
        return dofs, K, S

    # ------------------------------------------------------------------ assembly
    def _uncut_blocks(self, ref=False):
        """Yield (dofs (m,12), K (m,12,12), S (m,6,12), vox (m,)) per tet type for uncut tets
        (all tets and C = identity when ``ref``: the operator A0_11 of eq.
        constantCoefficientPreconditioner)."""
        for t in range(6):
            mask = np.ones(self.nvox, bool) if ref else ~self.cut[:, t]
            vox = np.flatnonzero(mask)
            if vox.size == 0:
                continue
            nodes = self.tet_nodes[vox, t]
            dofs = (np.arange(3)[None, None, :] * self.nFE + nodes[:, :, None]).reshape(-1, 12)
            B = self.B_std[t]
            vol = self.tet_vol[t]
            if ref:
                K = np.broadcast_to(vol * B.T @ B, (vox.size, 12, 12))
                S = np.broadcast_to(vol * B, (vox.size, 6, 12))
            else:
                ph = self.tet_phase[vox, t]
                lam = np.array([p[0] for p in self.phases])[ph] * self.scale[vox]
                mu = np.array([p[1] for p in self.phases])[ph] * self.scale[vox]
                Cl = iso_stiffness(1.0, 0.0)
                Cm = iso_stiffness(0.0, 1.0)
                Kl = vol * B.T @ Cl @ B
                Km = vol * B.T @ Cm @ B
                K = lam[:, None, None] * Kl + mu[:, None, None] * Km
                S = vol * (lam[:, None, None] * (Cl @ B) + mu[:, None, None] * (Cm @ B))
            yield dofs, K, S, vox

    def assemble(self):
        """Scaled system matrix A (eq. linearSystem via eq. linearSystem_element), the stress
        operator S (6 x ndof) with sum_e int C B u_e = S u (eq. Sapp_q) and
        Cbar = sum_e int C (6x6)."""
        rows, cols, vals = [], [], []
        Srows, Scols, Svals = [], [], []
        Cbar = np.zeros((6, 6))
        for dofs, K, S, vox in self._uncut_blocks():
            m = dofs.shape[0]
            rows.append(np.repeat(dofs, 12, axis=1).ravel())
            cols.append(np.tile(dofs, (1, 12)).ravel())
            vals.append(K.ravel())
            Srows.append(np.broadcast_to(np.arange(6)[None, :, None], (m, 6, 12)).ravel())
            Scols.append(np.broadcast_to(dofs[:, None, :], (m, 6, 12)).ravel())
            Svals.append(np.ascontiguousarray(S).ravel())
        for t in range(6):
            vox = np.flatnonzero(~self.cut[:, t])
            ph = self.tet_phase[vox, t]
            for p in range(self.nL + 1):
                sel = vox[ph == p]
                Cbar += self.tet_vol[t] * float(self.scale[sel].sum()) * iso_stiffness(*self.phases[p])
        for idx in range(len(self.cut_list)):
            dofs, K, S = self.cut_element(idx)
            rows.append(np.repeat(dofs, 24))
            cols.append(np.tile(dofs, 24))
            vals.append(K.ravel())
            Srows.append(np.repeat(np.arange(6), 24))
            Scols.append(np.tile(dofs, 6))
            Svals.append(S.ravel())
            v, t = self.cut_list[idx]
            _, sides = self.cut_data[idx]
            for s in (+1, -1):
                Cbar += float(sides[s][1].sum()) * self._C(self._side_phase(idx, s), v)
        A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(self.ndof, self.ndof)).tocsr()
        Sm = sp.coo_matrix((np.concatenate(Svals), (np.concatenate(Srows), np.concatenate(Scols))),
                           shape=(6, self.ndof)).tocsr()
        self.A, self.Sm, self.Cbar = A, Sm, Cbar
        return A, Sm, Cbar

    def assemble_reference(self):
        """A0_11 = int grad^s N_FE : grad^s N_FE (std DOFs only; eq. constantCoefficientPreconditioner)."""
        rows, cols, vals = [], [], []
        for dofs, K, S, vox in self._uncut_blocks(ref=True):
            rows.append(np.repeat(dofs, 12, axis=1).ravel())
            cols.append(np.tile(dofs, (1, 12)).ravel())
            vals.append(np.ascontiguousarray(K).ravel())
        n3 = 3 * self.nFE
        A0 = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                           shape=(n3, n3)).tocsr()
        self.A0 = A0
        return A0

    def rhs(self, eps):
        """b = sum_e Lambda_e^T int B^T C eps_bar (eq. b); the same element integral as the
        stress matrix of eq. Sapp_q, transposed: b = S^T eps_bar."""
        if not hasattr(self, "Sm"):
            self.assemble()
        return np.asarray(self.Sm.T @ np.asarray(eps, dtype=float)).ravel()

    # ------------------------------------------------------------------ solvers
    def _pinned_lu(self, A, nstd):
        """Sparse LU of A with the three std DOFs of node 0 removed.  The kernel of A is the
        translations of the standard part, so a pinned solution shifted to a zero std mean is
        the solution under the constraint sum_i u_FE^i = 0 (eq. X-FEM_space)."""
        keep = np.setdiff1d(np.arange(A.shape[0]), np.arange(3) * nstd)
        lu = spla.splu(A[keep][:, keep].tocsc(), permc_spec="MMD_AT_PLUS_A",
                       options={"SymmetricMode": True})

        def solve(rhs):
            x = np.zeros(A.shape[0])
            x[keep] = lu.solve(rhs[keep])
            for c in range(3):
                x[c * nstd:(c + 1) * nstd] -= x[c * nstd:(c + 1) * nstd].mean()
            return x
        return solve

    def solve_direct(self, eps):
        """Solve A u = -b with sum_i u_FE^i = 0 (eqs. discreteFormConti, X-FEM_space) by a
        sparse direct solve."""
        if not hasattr(self, "A"):
            self.assemble()
        if not hasattr(self, "_Alu"):
            self._Alu = self._pinned_lu(self.A, self.nFE)
        return self._Alu(-self.rhs(eps))

    def _green_sparse(self):
        if not hasattr(self, "_A0lu"):
            self._A0lu = self._pinned_lu(self.assemble_reference(), self.nFE)
        return self._A0lu

    def voxel_reference_matrix(self):
        """A0_11,v (24x24): the six tets' int grad^s N : grad^s N placed on the voxel's corner
        DOFs (eq. A0Voxel), with corners numbered as in the node table Y (Sec. 3) and DOFs
        node-major (3 * corner + component).  Uses the true tet volume h1 h2 h3 / 6."""
        Av = np.zeros((24, 24))
        corner_of = {tuple(c): k for k, c in enumerate(VOXEL_CORNERS)}
        for t in range(6):
            B = self.B_std[t]
            K = self.tet_vol[t] * B.T @ B
            idx = []
            for a in range(4):
                k = corner_of[tuple(self.tet_offsets[t][a])]
                idx.extend([3 * k, 3 * k + 1, 3 * k + 2])
            Av[np.ix_(idx, idx)] += K
        return Av

    def green_symbol(self):
        """Hermitian 3x3 matrices Z(xi)^H A0_v Z(xi) for every frequency (eq. GreenHermitian),
        Z = c(xi) (x) I_3 with c_j = exp(2 pi i sum_k Y_jk xi_k / N_k).  Shape (N1,N2,N3,3,3)."""
        Av = self.voxel_reference_matrix()
        n = self.n
        xi = np.meshgrid(*[np.fft.fftfreq(n[a]) for a in range(3)], indexing="ij")
        phase = sum(np.multiply.outer(xi[a], VOXEL_CORNERS[:, a]) for a in range(3))
        c = np.exp(2j * np.pi * phase)  # (N1,N2,N3,8)
        Z = np.einsum("...j,kl->...jkl", c, np.eye(3)).reshape(n + (24, 3))
        return np.einsum("...ai,ab,...bj->...ij", Z.conj(), Av, Z)

    def green_symbol_at(self, k):
        """The 3x3 matrix Z(xi)^H A0_v Z(xi) of eq. GreenHermitian at the single integer frequency
        k = (k1, k2, k3) (taken modulo the grid), without forming the full symbol array."""
        Av = self.voxel_reference_matrix()
        xi = np.array([np.fft.fftfreq(self.n[a])[int(k[a]) % self.n[a]] for a in range(3)])
        c = np.exp(2j * np.pi * (VOXEL_CORNERS @ xi))  # (8,)
        Z = np.kron(c[:, None], np.eye(3))  # (24, 3), DOFs node-major
        return Z.conj().T @ Av @ Z

    def precondition_modes(self, modes):
        """P^{-1} (std part, eq. GreenHermitian) of the real field f = sum_m Re(a_m e^{2 pi i
        k_m . x / N}) given as a list of (k_m, a_m) with a_m a complex 3-vector: since the Green
        operator is diagonal in Fourier space with M(-xi) = conj M(xi), the result is
        z = sum_m Re(M(k_m)^{-1} a_m e^{2 pi i k_m . x / N}) (the zero frequency maps to 0).
        Returns (f, z), each of length 3 N (component-major)."""
        n = self.n
        i, j, k = np.meshgrid(*[np.arange(n[a]) for a in range(3)], indexing="ij")
        f = np.zeros((3,) + n)
        z = np.zeros((3,) + n)
        for kv, a in modes:
            kv = [int(v) % n[q] for q, v in enumerate(kv)]
            a = np.asarray(a, dtype=complex)
            ph = np.exp(2j * np.pi * (kv[0] * i / n[0] + kv[1] * j / n[1] + kv[2] * k / n[2]))
            if kv == [0, 0, 0]:
                b = np.zeros(3, dtype=complex)
            else:
                b = np.linalg.solve(self.green_symbol_at(kv), a)
            for q in range(3):
                f[q] += np.real(a[q] * ph)
                z[q] += np.real(b[q] * ph)
        return f.ravel(), z.ravel()

    def _green_fft(self):
        Mx = self.green_symbol()
        Mx[0, 0, 0] = np.eye(3)
        Minv = np.linalg.inv(Mx)
        Minv[0, 0, 0] = 0.0
        n = self.n

        def apply(f):
            F = np.fft.fftn(f.reshape((3,) + n), axes=(1, 2, 3))
            G = np.einsum("...ij,j...->i...", Minv, F)
            return np.real(np.fft.ifftn(G, axes=(1, 2, 3))).ravel()
        return apply

    def _enr_precondition(self, fX, enr):
        """Enriched part of P^{-1}: the identity on the scaled DOFs (eq. scaledPreconditioner,
        the paper's choice) or, for enr="block3", the inverse of each enriched node's 3x3 block
        of the scaled reference Gram matrix (a variant, not in the paper).  fX is component-major
        (3, nX) flattened."""
        if enr == "identity":
            return fX.copy()
        if enr != "block3":
            raise ValueError(enr)
        F = fX.reshape(3, self.nX).T  # (nX, 3)
        Z = np.linalg.solve(self.Bblk, F[:, :, None])[:, :, 0]
        return Z.T.ravel()

    def precondition(self, f, green="sparse", enr="identity"):
        """z = P^{-1} f with P = diag(A0_11, I) (eq. scaledPreconditioner); enr="block3" uses the
        node blocks of the enriched reference Gram matrix instead of I."""
        n3 = 3 * self.nFE
        g = self._green_sparse() if green == "sparse" else self._green_fft()
        z = np.empty_like(f)
        z[:n3] = g(f[:n3])
        z[n3:] = self._enr_precondition(f[n3:], enr)
        return z

    def mean_stress(self, u, eps):
        """<sigma>_Y = (1/|Y|) sum_e int C (eps_bar + grad^s u) (reading of eq. Sapp_q)."""
        if not hasattr(self, "Sm"):
            self.assemble()
        return (np.asarray(self.Sm @ u).ravel() + self.Cbar @ np.asarray(eps, float)) / self.volY

    def basic_step(self):
        """Step size s0 = 2 / (C_- + C_+) of the basic scheme (eq. stepsize): C_- (C_+) is the
        smallest (largest) eigenvalue of the stiffness tensors of all materials; with isotropic
        phases the eigenvalues are 2 mu and 3 lambda + 2 mu, times the extreme voxel scales."""
        ev = [e for lam, mu in self.phases for e in (2.0 * mu, 3.0 * lam + 2.0 * mu)]
        return 2.0 / (min(ev) * float(self.scale.min()) + max(ev) * float(self.scale.max()))

    def pcg(self, eps, tol=1e-10, maxit=10000, green="sparse", u0=None, enr="identity",
            scheme="cg", step=None, bb_rule="bb1", bb_cycle=1):
        """Linear CG of Algorithm 1 on A u = -b with the X-FFT preconditioner.

        Reading of Algorithm 1: f is the negative residual -b - A u, z = A d is the linear part
        of the residual map, alpha = res_old^2 / <z, d>, u += alpha d, f -= alpha z, and the
        loop stops once sqrt(f^T P^{-1} f / |Y|) <= tol ||<sigma(u)>_Y|| (eqs.
        stoppingCriterion, convergence; the 1/|Y| makes both sides stresses) or after maxit
        iterations.  Returns (u, info) with iteration count and residual history.

        The other schemes of Sec. 2.3 on the same system and preconditioner: "basic" (fixed
        step s0 of eq. stepsize, beta = 0), "bb" (Barzilai-Borwein, beta = 0, s0 first) and
        "nlcg" (nonlinear CG: fixed step s0, no line search, Fletcher-Reeves beta = res^2 /
        res_old^2).  The paper cites the Barzilai-Borwein scheme without its formula; with
        du = u_k - u_{k-1} and dg = A du (the change of the energy gradient) the classical
        steps are ``bb_rule`` "bb1" = <du, P du> / <du, dg> and "bb2" = <du, dg> /
        <dg, P^{-1} dg> in the metric of the preconditioner, "alt" (bb2 and bb1 in turn, bb2
        on odd iterations), "bb1e" = <du, du> / <du, dg> and "bb2e" = <du, dg> / <dg, dg> in
        the Euclidean metric of the scaled DOFs; ``bb_cycle`` m renews the step every m
        iterations and keeps it in between (cyclic Barzilai-Borwein).
        """
        if not hasattr(self, "A"):
            self.assemble()
        gfun = self._green_sparse() if green == "sparse" else self._green_fft()
        n3 = 3 * self.nFE
        if scheme not in ("cg", "basic", "bb", "nlcg"):
            raise ValueError(scheme)
        if bb_rule not in ("bb1", "bb2", "alt", "bb1e", "bb2e") or int(bb_cycle) < 1:
            raise ValueError(bb_rule)
        s0 = self.basic_step() if step is None else float(step)
        alpha = s0
        du = dg = None

        def P(f):
            z = np.empty_like(f)
            z[:n3] = gfun(f[:n3])
            z[n3:] = self._enr_precondition(f[n3:], enr)
            return z

        b = self.rhs(eps)
        u = np.zeros(self.ndof) if u0 is None else np.array(u0, dtype=float)
        f = -b - self.A @ u
        d = P(f)
        rr = float(f @ d)
        hist = []
        k = 0
        converged = False
        while True:
            res = math.sqrt(max(rr, 0.0) / self.volY)
            sig = np.linalg.norm(self.mean_stress(u, eps))
            hist.append(res / sig if sig > 0 else res)
            if res <= tol * sig:
                converged = True
                break
            if k >= maxit:
                break
            z = self.A @ d
            if scheme == "cg":
                alpha = rr / float(z @ d)  # exact line search along d
            elif scheme in ("basic", "nlcg"):  # fixed step s0 (no line search)
                alpha = s0
            elif k == 0:
                alpha = s0
            elif (k - 1) % int(bb_cycle) == 0:  # Barzilai-Borwein step from du, dg
                rule = bb_rule if bb_rule != "alt" else ("bb2" if k % 2 == 1 else "bb1")
                if rule == "bb1":
                    alpha = float(du @ self._precond_metric(du, enr)) / float(du @ dg)
                elif rule == "bb2":
                    alpha = float(du @ dg) / float(dg @ P(dg))
                elif rule == "bb1e":
                    alpha = float(du @ du) / float(du @ dg)
                else:
                    alpha = float(du @ dg) / float(dg @ dg)
            du = alpha * d
            dg = alpha * z
            u += alpha * d
            f -= alpha * z
            zz = P(f)
            rr_new = float(f @ zz)
            # Fletcher-Reeves momentum for linear and nonlinear CG; none for basic / BB
            beta = rr_new / rr if scheme in ("cg", "nlcg") else 0.0
            d = zz + beta * d
            rr = rr_new
            k += 1
        return u, {"iters": k, "converged": converged, "history": hist}

    def _precond_metric(self, du, enr="identity"):
        """P du for the metric of the preconditioner, P itself (not its inverse):
        P = diag(A0_11, I) (eq. scaledPreconditioner) with the assembled A0_11 on the standard
        part and the identity (or, for enr="block3", the enriched node blocks) on the scaled
        enriched part."""
        if not hasattr(self, "A0"):
            self.assemble_reference()
        n3 = 3 * self.nFE
        out = du.copy()
        out[:n3] = self.A0 @ du[:n3]
        if enr == "block3":
            F = du[n3:].reshape(3, self.nX).T
            out[n3:] = np.einsum("jkl,jl->jk", self.Bblk, F).T.ravel()
        return out

    # ------------------------------------------------------------------ post-processing
    def effective_stiffness(self, solver="direct", tol=1e-12, green="sparse"):
        """C_eff column k = <sigma> for eps_bar = E_k (Mandel basis) and the energy form
        C_kl = (1/|Y|) int eps_k : C : eps_l.  Returns (C_stress, C_energy, U) with U the
        6 solution vectors."""
        if not hasattr(self, "A"):
            self.assemble()
        U = []
        Cs = np.zeros((6, 6))
        for k in range(6):
            e = np.eye(6)[k]
            u = self.solve_direct(e) if solver == "direct" else self.pcg(e, tol=tol, green=green)[0]
            U.append(u)
            Cs[:, k] = self.mean_stress(u, e)
        U = np.array(U)
        SU = np.asarray(self.Sm @ U.T)  # (6, 6): column l = S u_l
        AU = np.asarray(self.A @ U.T)
        Ce = (self.Cbar + SU + SU.T + U @ AU) / self.volY
        return Cs, Ce, U

    def voxel_stress(self, u, eps):
        """Per-voxel average stress (1/|v|) int_v C (eps_bar + grad^s u), shape (nvox, 6)."""
        eps = np.asarray(eps, float)
        out = np.zeros((self.nvox, 6))
        for dofs, K, S, vox in self._uncut_blocks():
            out[vox] += np.einsum("mrk,mk->mr", S, u[dofs])
        for t in range(6):
            vox = np.flatnonzero(~self.cut[:, t])
            ph = self.tet_phase[vox, t]
            for p in range(self.nL + 1):
                sel = vox[ph == p]
                out[sel] += (self.tet_vol[t] * self.scale[sel])[:, None] * (iso_stiffness(*self.phases[p]) @ eps)[None, :]
        for idx in range(len(self.cut_list)):
            dofs, K, S = self.cut_element(idx)
            v, t = self.cut_list[idx]
            _, sides = self.cut_data[idx]
            out[v] += S @ u[dofs]
            for s in (+1, -1):
                out[v] += float(sides[s][1].sum()) * (self._C(self._side_phase(idx, s), v) @ eps)
        return out / float(np.prod(self.h))

    # ------------------------------------------------------------------ gradient
    def _strains_uncut(self, U, t, vox):
        """Mandel strains (nrhs, m, 6) of tet type t in voxels vox for solution vectors U
        (without the macroscopic part)."""
        nodes = self.tet_nodes[vox, t]
        dofs = (np.arange(3)[None, None, :] * self.nFE + nodes[:, :, None]).reshape(-1, 12)
        return np.einsum("rk,nmk->nmr", self.B_std[t], U[:, dofs])

    def stiffness_gradient(self, U, E=None):
        """Derivatives of the energy-form C_eff with respect to the phase Lame constants and
        the per-voxel scale: dC_kl/dtheta = (1/|Y|) int eps_k : dC/dtheta : eps_l with
        eps_k = E_k + grad^s u_k (envelope identity; the basis does not depend on C).

        Returns (dC_dlame (2(K+1),6,6) in order lam_0, mu_0, lam_1, mu_1, ... (one interface:
        lam_minus, mu_minus, lam_plus, mu_plus); dC_ds (nvox,6,6)).
        """
        E = np.eye(6) if E is None else np.asarray(E, float)
        nr = U.shape[0]
        nph = self.nL + 1
        Al = [np.zeros((self.nvox, nr, nr)) for _ in range(nph)]  # int tr eps_k tr eps_l
        Am = [np.zeros((self.nvox, nr, nr)) for _ in range(nph)]  # int 2 eps_k : eps_l
        m = np.array([1.0, 1.0, 1.0, 0.0, 0.0, 0.0])
        for t in range(6):
            vox = np.flatnonzero(~self.cut[:, t])
            if vox.size == 0:
                continue
            eps = self._strains_uncut(U, t, vox) + E[:, None, :]  # (nr, m, 6)
            tr = eps @ m
            ph = self.tet_phase[vox, t]
            vol = self.tet_vol[t]
            al = vol * np.einsum("km,lm->mkl", tr, tr)
            am = 2.0 * vol * np.einsum("kmr,lmr->mkl", eps, eps)
            for p in range(nph):
                sel = ph == p
                np.add.at(Al[p], vox[sel], al[sel])
                np.add.at(Am[p], vox[sel], am[sel])
        for idx in range(len(self.cut_list)):
            v, t = self.cut_list[idx]
            Lv, sides = self.cut_data[idx]
            G = self.tet_grads[t]
            nodes = self.tet_nodes[v, t]
            eids = self.enr_id[nodes]
            dofs = np.concatenate([
                (np.arange(3)[None, :] * self.nFE + nodes[:, None]).ravel(),
                (3 * self.nFE + np.arange(3)[None, :] * self.nX + eids[:, None]).ravel()])
            scale = np.concatenate([np.ones(12), self.Dinvsqrt[eids].ravel()])
            ue = U[:, dofs] * scale  # (nr, 24)
            for s in (+1, -1):
                bary, w = sides[s]
                BX = self._enriched_B(G, Lv, s, bary)
                Bf = np.concatenate([np.broadcast_to(self.B_std[t], BX.shape), BX], axis=2)
                eps = np.einsum("qrj,nj->nqr", Bf, ue) + E[:, None, :]
                tr = eps @ m
                p = self._side_phase(idx, s)
                Al[p][v] += np.einsum("q,kq,lq->kl", w, tr, tr)
                Am[p][v] += 2.0 * np.einsum("q,kqr,lqr->kl", w, eps, eps)
        sc = self.scale[:, None, None]
        dl = np.stack([x for p in range(nph) for x in ((sc * Al[p]).sum(0), (sc * Am[p]).sum(0))])
        ds = sum(self.phases[p][0] * Al[p] + self.phases[p][1] * Am[p] for p in range(nph))
        return dl / self.volY, ds / self.volY

    # ------------------------------------------------------------------ local evaluation
    def apply(self, d, eps=None):
        """A d (+ b if eps given): the residual map of eq. resVector up to the sign reading."""
        if not hasattr(self, "A"):
            self.assemble()
        out = np.asarray(self.A @ d).ravel()
        if eps is not None:
            out += self.rhs(eps)
        return out
