"""Frequency weights: generalized tetrahedron x(k) and plain Lorentzian X (oracle).

Eq. Xakqbk (time-ordered):  X = 1/(w - D + i d) - 1/(w + D - i d),  D = E_{a,k+q} - E_{b,k}.
Both terms have the form 1/(z - D):  z1 = w + i d,  z2 = -w + i d
(retarded variant: z2 = -w - i d, for which chi(-w) = chi(w)^*).  On the
imaginary axis w = i nu.

Eq. tetrahedron: X is replaced by vertex weights x(k) of a Brillouin-zone
integration (generalized tetrahedron method, refs. Fujiwara 2003 and Nohara
2009).  The paper prints no formula; the reading implemented here:

  * each sub-cell of the Gamma-centred mesh is cut into 6 tetrahedra that
    share its shortest main diagonal (volume V_BZ / (6 N_k) each);
  * D(k) and the matrix-element product are interpolated linearly over a
    tetrahedron (barycentric weights lambda_j at vertex j);
  * the resonant factor 1/(z - D) is integrated exactly.  With the
    Hermite-Genocchi formula,
        (1/V_t) int_t lambda_j / (z - D(k)) dk = f_z[d1, d2, d3, d4, d_j],
    the fourth-order divided difference (node j repeated) of
        f_z(x) = (z - x)^3 log(z - x),
    whose fourth derivative is 6 / (z - x);
  * vertex weight x(k) = (1/6) sum over the 24 tetrahedra t that contain k
    of [f_z1 + f_z2][nodes of t, d_{j(k)}]; then (1/N_k) sum_k x(k) F(k)
    is the Brillouin-zone average and x(k) = 1 for a constant integrand 1.

Degeneracy parameters delta_a, delta_r (Eq. tetrahedron): after sorting, a
node joins the group of the preceding node when it lies closer than
delta_a + delta_r * max(|x_start|, |x_i|) to the group's first node; all
nodes of a group are replaced by the group mean (confluent limit).

Evaluating a divided difference by the textbook recursion loses digits when
a run of nodes is narrow compared with its distance to the pole z.  Such runs
(spread <= TAU |z - c|, c the run's midpoint) are evaluated instead with the
Taylor-series identity for the divided difference of an analytic function,
    f[x_i..x_j] = sum_{m >= n} f^(m)(c)/m! * h_{m-n}(x_i - c, ..., x_j - c),
h_k being the complete homogeneous symmetric polynomial.  Both branches are
exact identities; the switch only picks the stable one.
"""
import numpy as np

from .lattice import kmesh_index

TAU = 0.5
NTERMS = 40


def tetrahedra(kmesh, recip):
    """[6 N_k, 4] mesh indices of the tetrahedra (shortest main diagonal)."""
    n = np.asarray(kmesh, dtype=np.int64)
    recip = np.asarray(recip, dtype=np.float64)
    starts = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1)]
    best_len, best_s = None, None
    for s in starts:
        d = (1.0 - 2.0 * np.array(s)) / n
        ln = float(np.linalg.norm(d @ recip))
        if best_len is None or ln < best_len * (1.0 - 1e-12):
            best_len, best_s = ln, np.array(s)
    perms = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]
    offs = []
    for (i, j, _k) in perms:
        v0 = np.zeros(3, dtype=np.int64)
        v1 = v0.copy(); v1[i] = 1
        v2 = v1.copy(); v2[j] = 1
        v3 = np.ones(3, dtype=np.int64)
        offs.append([v0, v1, v2, v3])
    offs = np.array(offs)
    offs = np.where(best_s[None, None, :] == 1, 1 - offs, offs)
    out = []
    for i1 in range(n[0]):
        for i2 in range(n[1]):
            for i3 in range(n[2]):
                base = np.array([i1, i2, i3])
                for t in range(6):
                    out.append([kmesh_index(n, base + offs[t, v]) for v in range(4)])
    return np.array(out, dtype=np.int64)


def _b_coeff(m, logy):
    """f^(m)(c)/m! = (z-c)^(3-m) * b_m  for f(x) = (z-x)^3 log(z-x)."""
    if m == 0:
        return logy
    if m == 1:
        return -(3.0 * logy + 1.0)
    if m == 2:
        return (6.0 * logy + 5.0) / 2.0
    if m == 3:
        return -(6.0 * logy + 11.0) / 6.0
    return np.full_like(logy, 6.0 / (m * (m - 1) * (m - 2) * (m - 3)))


def merge_nodes(x, delta_a, delta_r):
    """Sort nodes along the last axis and replace degenerate groups by their mean."""
    x = np.sort(np.asarray(x, dtype=np.float64), axis=-1)
    p = x.shape[-1]
    gid = np.zeros(x.shape, dtype=np.int64)
    start = x[..., 0].copy()
    for i in range(1, p):
        thr = delta_a + delta_r * np.maximum(np.abs(start), np.abs(x[..., i]))
        new = (x[..., i] - start) >= thr
        gid[..., i] = gid[..., i - 1] + new
        start = np.where(new, x[..., i], start)
    out = np.empty_like(x)
    for g in range(p):
        mask = gid == g
        cnt = mask.sum(axis=-1, keepdims=True)
        mean = np.where(cnt > 0, (x * mask).sum(axis=-1, keepdims=True) / np.maximum(cnt, 1), 0.0)
        out = np.where(mask, mean, out)
    return out


def divided_difference(nodes, z, delta_a=0.0, delta_r=0.0):
    """f_z[x_0, ..., x_n] for f_z(x) = (z-x)^3 log(z-x); nodes [..., n+1], z broadcastable."""
    x = merge_nodes(nodes, delta_a, delta_r)
    z = np.asarray(z, dtype=np.complex128)
    p = x.shape[-1]
    shape = np.broadcast_shapes(x.shape[:-1], z.shape)
    x = np.broadcast_to(x, shape + (p,))
    z = np.broadcast_to(z, shape)
    table = {}
    for i in range(p):
        y = z - x[..., i]
        table[(i, i)] = y ** 3 * np.log(y)
    for n in range(1, p):
        for i in range(0, p - n):
            j = i + n
            s = x[..., j] - x[..., i]
            c = 0.5 * (x[..., i] + x[..., j])
            yc = z - c
            use_series = s <= TAU * np.abs(yc)
            rec = (table[(i + 1, j)] - table[(i, j - 1)]) / np.where(s > 0, s, 1.0)
            # series:  yc^(3-n) * sum_{m=n}^{n+NTERMS} b_m * h_{m-n}((x - c)/yc)
            logy = np.log(yc)
            h = [np.ones(shape, dtype=np.complex128)] + [np.zeros(shape, dtype=np.complex128)] * NTERMS
            for v in range(i, j + 1):
                u = (x[..., v] - c) / yc
                for k in range(1, NTERMS + 1):
                    h[k] = h[k] + u * h[k - 1]
            acc = np.zeros(shape, dtype=np.complex128)
            for k in range(NTERMS + 1):
                acc = acc + _b_coeff(n + k, logy) * h[k]
            ser = yc ** (3 - n) * acc
            table[(i, j)] = np.where(use_series, ser, rec)
    return table[(0, p - 1)]


def poles(freq, axis, delta, ordering):
    """(z1, z2) per frequency, Eq. Xakqbk with w real or w = i nu."""
    w = np.asarray(freq, dtype=np.float64).astype(np.complex128)
    if axis == "imag":
        w = 1j * w
    elif axis != "real":
        raise ValueError(axis)
    z1 = w + 1j * delta
    if ordering == "time":
        z2 = -w + 1j * delta
    elif ordering == "retarded":
        z2 = -w - 1j * delta
    else:
        raise ValueError(ordering)
    if np.any(np.abs(z1.imag) == 0) or np.any(np.abs(z2.imag) == 0):
        raise ValueError("a pole lies on the real axis")
    return z1, z2


def vertex_weights(e_occ, e_emp_kq, tets, z1, z2, delta_a, delta_r, k_list=None, chunk=64):
    """x[k, a, o, f] (Eq. tetrahedron), for the k in k_list (default: all)."""
    nk, nocc = e_occ.shape
    nemp = e_emp_kq.shape[1]
    nf = len(z1)
    ks = np.arange(nk) if k_list is None else np.asarray(k_list)
    want = np.zeros(nk, dtype=bool)
    want[ks] = True
    sel = tets[np.any(want[tets], axis=1)]
    x = np.zeros((nk, nemp, nocc, nf), dtype=np.complex128)
    zz = [np.asarray(z1)[None, None, None, :], np.asarray(z2)[None, None, None, :]]
    for c0 in range(0, len(sel), chunk):
        tt = sel[c0:c0 + chunk]                                  # [T, 4]
        d = e_emp_kq[tt][:, :, :, None] - e_occ[tt][:, :, None, :]   # [T, 4, nemp, nocc]
        d = d[..., None]                                          # [T, 4, nemp, nocc, 1]
        for j in range(4):
            rows = np.nonzero(want[tt[:, j]])[0]
            if len(rows) == 0:
                continue
            dj = d[rows]
            nodes = np.stack([dj[:, 0], dj[:, 1], dj[:, 2], dj[:, 3], dj[:, j]], axis=-1)  # [T',nemp,nocc,1,5]
            val = sum(divided_difference(nodes, z, delta_a, delta_r) for z in zz)        # [T',nemp,nocc,nf]
            for r, t in enumerate(rows):
                x[tt[t, j]] += val[r] / 6.0
    return x[ks]


def clip_negative(e):
    """Sub-tetrahedra of the part of a tetrahedron where a function linear on it is negative.

    e: [4] values at the vertices.  Returns a list of [4, 4] matrices B whose row i is sub-vertex i
    in barycentric coordinates of the tetrahedron (so a sub-vertex is sum_j B[i, j] vertex_j, and
    the sub-tetrahedron's volume is |det B| of the whole).  With n vertices below zero the region
    is: nothing (n = 0); the corner at the lowest vertex cut off by the zero plane (n = 1); a
    triangular prism between the two low vertices and the plane (n = 2); the whole minus the
    corner at the highest vertex, again a prism (n = 3); the whole (n = 4).  A prism with
    triangles A, B and lateral edges A_i B_i is cut into (A0 A1 A2 B0), (A1 A2 B0 B1), (A2 B0 B1 B2).
    Zero counts as not negative (the boundary has no volume)."""
    e = np.asarray(e, dtype=np.float64)
    s = np.argsort(e, kind="stable")
    n = int(np.sum(e < 0.0))
    eye = np.eye(4)

    def cut(u, v):
        # the point of edge u-v where the function vanishes (e[u] < 0 <= e[v])
        t = e[u] / (e[u] - e[v])
        return (1.0 - t) * eye[u] + t * eye[v]

    def prism(A, B):
        return [np.array([A[0], A[1], A[2], B[0]]), np.array([A[1], A[2], B[0], B[1]]),
                np.array([A[2], B[0], B[1], B[2]])]

    if n == 0:
        return []
    if n == 4:
        return [eye.copy()]
    if n == 1:
        return [np.array([eye[s[0]], cut(s[0], s[1]), cut(s[0], s[2]), cut(s[0], s[3])])]
    if n == 2:
        return prism([eye[s[0]], cut(s[0], s[2]), cut(s[0], s[3])],
                     [eye[s[1]], cut(s[1], s[2]), cut(s[1], s[3])])
    return prism([eye[s[0]], eye[s[1]], eye[s[2]]],
                 [cut(s[0], s[3]), cut(s[1], s[3]), cut(s[2], s[3])])


def occupied_pieces(eo, ea, fermi):
    """Sub-tetrahedra (barycentric [4, 4] matrices of the whole) of the part of a tetrahedron where
    the occupied band lies below the Fermi energy and the empty band at k+q above it: eo, ea [4]
    vertex energies, each interpolated linearly (Fermi-surface clipping of the metallic
    generalized tetrahedron method)."""
    out = []
    for B in clip_negative(np.asarray(eo) - fermi):
        # the empty band's values at this piece's vertices; keep where it lies above the Fermi energy
        g = B @ (fermi - np.asarray(ea))
        for C in clip_negative(g):
            out.append(C @ B)
    return out


def piece_vertex_weights(F, d, sub_weight):
    """Contributions of pieces of a tetrahedron to its four vertices: for a piece with barycentric
    matrix F (volume |det F| of the whole) and D linear with vertex values d, lambda_j = sum_i mu_i
    F[i, j] (mu_i the piece's own barycentric weights), so the piece adds |det F| sum_i F[i, j] w_i
    to vertex j, w_i its vertex-i weight (the unclipped formula on the piece).
    F [P, 4, 4], d [P, 4] (D at the tetrahedron's vertices, per piece); sub_weight(ds) takes D at
    the pieces' vertices [P, 4] and returns their vertex weights [P, 4, ...].  Returns [P, 4, ...]."""
    vol = np.abs(np.linalg.det(F))                          # [P]
    ds = np.einsum("pij,pj->pi", F, d)                      # [P, 4]
    w = np.asarray(sub_weight(ds))                          # [P, 4 (i), ...]
    return np.einsum("p,pij,pi...->pj...", vol, F, w)


def clipped_vertex_weights(d, pieces, sub_weight):
    """(1/V_t) int over the pieces of lambda_j g(D) for the four vertices j of a tetrahedron (D
    linear, vertex values d [4]): the sum of piece_vertex_weights.  Returns [4, ...], or None
    without pieces."""
    if not pieces:
        return None
    F = np.stack(pieces)
    d = np.broadcast_to(np.asarray(d, dtype=np.float64), (len(pieces), 4))
    return piece_vertex_weights(F, d, sub_weight).sum(axis=0)


def metal_vertex_weights(e_occ, e_emp_kq, tets, z1, z2, delta_a, delta_r, fermi, k_list=None):
    """x[k, a, o, f] of the metallic generalized tetrahedron method: as vertex_weights, but each
    tetrahedron contributes only over its part where band o (at k) is occupied and band a (at
    k + q) is empty, with the Fermi energy `fermi` (both bands interpolated linearly).  The pieces
    of all pairs of one tetrahedron are evaluated together."""
    nk, nocc = e_occ.shape
    nemp = e_emp_kq.shape[1]
    nf = len(z1)
    ks = np.arange(nk) if k_list is None else np.asarray(k_list)
    want = np.zeros(nk, dtype=bool)
    want[ks] = True
    sel = tets[np.any(want[tets], axis=1)]
    x = np.zeros((nk, nemp, nocc, nf), dtype=np.complex128)
    zz = [np.asarray(z1)[None, None, :], np.asarray(z2)[None, None, :]]

    def sub_weight(ds):
        # nodes of piece p, vertex i: its four D values and D_i again -> [P, 4, 1, 5]
        nodes = np.concatenate([np.repeat(ds[:, None, :], 4, axis=1), ds[:, :, None]], axis=2)[:, :, None, :]
        return sum(divided_difference(nodes, z, delta_a, delta_r) for z in zz)    # [P, 4, nf]

    for tt in sel:
        F, d, owner = [], [], []
        for a in range(nemp):
            for o in range(nocc):
                eo, ea = e_occ[tt, o], e_emp_kq[tt, a]
                for B in occupied_pieces(eo, ea, fermi):
                    F.append(B)
                    d.append(ea - eo)
                    owner.append((a, o))
        if not F:
            continue
        contrib = piece_vertex_weights(np.stack(F), np.stack(d), sub_weight)     # [P, 4, nf]
        val = np.zeros((nemp, nocc, 4, nf), dtype=np.complex128)
        own = np.array(owner)
        np.add.at(val, (own[:, 0], own[:, 1]), contrib)
        for j in range(4):
            if want[tt[j]]:
                x[tt[j]] += val[:, :, j] / 6.0
    return x[ks]


def lorentz_x(e_occ, e_emp_kq, z1, z2):
    """X of Eq. Xakqbk at the mesh points themselves: [k, a, o, f]."""
    d = (e_emp_kq[:, :, None] - e_occ[:, None, :])[..., None]
    return 1.0 / (np.asarray(z1) - d) + 1.0 / (np.asarray(z2) - d)
