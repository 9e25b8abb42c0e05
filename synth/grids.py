"""Seeded Cartesian meshes, permeability fields and boundary data (no solver arithmetic here).

The cell graph follows the paper's finite-volume setting (Sec. 2.1): one pressure unknown per cell, one flux per
interface, interior interfaces stored once with K < L, boundary interfaces carrying either a prescribed pressure
(Dirichlet) or a prescribed normal flux (Neumann). The geometric half transmissibility of a cell towards an interface
(eq. half-transmissibility) is |eps| K_0 / dist(x_K, x_eps) for a scalar K_0 on an orthogonal grid, whose collocation
point is the face centre (Remark on collocation points).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

BC_INTERIOR, BC_DIRICHLET, BC_NEUMANN = 0, 1, 2
KAPPA_EXP, KAPPA_INV1P2, KAPPA_RICHARDS = 0, 1, 2


@dataclass
class Mesh:
    """A cell graph with geometric data; every array is a plain numpy array in the layout the C ABI takes."""
    n_cells: int
    cell_volume: np.ndarray          # [N] float64
    face_cells: np.ndarray           # [F, 2] int32, K < L, L = -1 on boundary faces
    half_trans: np.ndarray           # [F, 2] float64, (Ups_K, Ups_L); Ups_L = 0 on boundary faces
    face_bc: np.ndarray              # [F] uint8: 0 interior, 1 Dirichlet, 2 Neumann
    face_area: np.ndarray            # [F] float64
    shape: tuple = ()
    perm: np.ndarray | None = None   # [N] K_0 per cell (for reference only)

    @property
    def n_faces(self) -> int:
        return int(self.face_cells.shape[0])


def _lin(shape):
    return np.arange(int(np.prod(shape)), dtype=np.int64).reshape(shape[::-1]).T  # index = i + nx*(j + ny*k)


def cartesian_mesh(shape, K, dirichlet_x=True, lengths=None, dirichlet_axes=None):
    """Unit square/cube (or a box of the given side lengths) split into shape cells; K is [N] in lexicographic order
    (x fastest).

    Boundary faces on x = 0 and x = 1 are Dirichlet, all others Neumann (no-flow unless data says otherwise);
    dirichlet_axes, if given, lists the axes whose two boundary sides are Dirichlet instead.
    """
    shape = tuple(int(s) for s in shape)
    d = len(shape)
    lengths = [1.0] * d if lengths is None else [float(v) for v in lengths]
    h = np.array([lengths[i] / s for i, s in enumerate(shape)])
    idx = _lin(shape)
    N = idx.size
    vol = np.full(N, float(np.prod(h)))
    K = np.asarray(K, dtype=np.float64).reshape(-1)
    fc, ht, bc, area = [], [], [], []
    for ax in range(d):
        a_face = float(np.prod(np.delete(h, ax)))
        dist = h[ax] / 2.0
        lo = np.take(idx, np.arange(shape[ax] - 1), axis=ax).reshape(-1, order="F")
        hi = np.take(idx, np.arange(1, shape[ax]), axis=ax).reshape(-1, order="F")
        order = np.argsort(lo, kind="stable")
        lo, hi = lo[order], hi[order]
        fc.append(np.stack([lo, hi], 1))
        ht.append(np.stack([a_face * K[lo] / dist, a_face * K[hi] / dist], 1))
        bc.append(np.zeros(lo.size, np.uint8))
        area.append(np.full(lo.size, a_face))
    for ax in range(d):
        a_face = float(np.prod(np.delete(h, ax)))
        dist = h[ax] / 2.0
        for side in (0, shape[ax] - 1):
            cells = np.sort(np.take(idx, side, axis=ax).reshape(-1))
            fc.append(np.stack([cells, np.full(cells.size, -1)], 1))
            ht.append(np.stack([a_face * K[cells] / dist, np.zeros(cells.size)], 1))
            dir_here = (ax in dirichlet_axes) if dirichlet_axes is not None else (ax == 0 and dirichlet_x)
            kind = BC_DIRICHLET if dir_here else BC_NEUMANN
            bc.append(np.full(cells.size, kind, np.uint8))
            area.append(np.full(cells.size, a_face))
    return Mesh(n_cells=N, cell_volume=vol,
                face_cells=np.concatenate(fc).astype(np.int32),
                half_trans=np.concatenate(ht).astype(np.float64),
                face_bc=np.concatenate(bc), face_area=np.concatenate(area), shape=shape, perm=K)


def voronoi_mesh(n_side, K_of_points, seed=3, jitter=0.4):
    """Clipped 3D Voronoi tessellation of a jittered n_side^3 lattice in the unit cube (an unstructured cell graph).

    Points x_K = lattice centres + U(-jitter, jitter) h. The cube clips the cells by mirroring the points within three
    lattice spacings of each of its six faces across that face: a ridge between a point and its own mirror is a
    boundary face. Faces smaller than 1e-8 h^2 (slivers of the tessellation's round-off) are dropped. Interior faces bisect the K-L segment, so the collocation point is the midpoint and
    Ups_bar = |eps| K_0 / (d_KL / 2); boundary faces use the distance to the face. A cell's volume is the sum of the
    pyramids from its point over its faces (|eps| d / 6 each, the point lying inside its own convex cell). Faces on
    x = 0 and x = 1 are Dirichlet, the rest Neumann. K_of_points(points) gives K_0 per cell.
    """
    from scipy.spatial import Voronoi
    rng = np.random.default_rng(seed)
    h = 1.0 / n_side
    g1 = (np.arange(n_side) + 0.5) * h
    P = np.stack(np.meshgrid(g1, g1, g1, indexing="ij"), -1).reshape(-1, 3)
    P = np.clip(P + rng.uniform(-jitter, jitter, P.shape) * h, 1e-6, 1 - 1e-6)
    n = P.shape[0]
    mirrors, owner, mface = [], [], []
    for ax in range(3):
        for side in (0.0, 1.0):
            sel = np.where(np.abs(P[:, ax] - side) < 3.0 * h)[0]
            Q = P[sel].copy()
            Q[:, ax] = 2 * side - Q[:, ax]
            mirrors.append(Q)
            owner.append(sel)
            mface.append(np.full(sel.size, 2 * ax + int(side)))
    allp = np.concatenate([P] + mirrors)
    owner = np.concatenate(owner)
    mface = np.concatenate(mface)
    vor = Voronoi(allp)
    K = np.asarray(K_of_points(P), dtype=np.float64)
    rp = np.asarray(vor.ridge_points)
    lens = np.fromiter((len(r) for r in vor.ridge_vertices), dtype=np.int64, count=len(vor.ridge_vertices))
    flat = np.fromiter((v for r in vor.ridge_vertices for v in r), dtype=np.int64, count=int(lens.sum()))
    start = np.concatenate([[0], np.cumsum(lens)[:-1]])
    has_inf = np.zeros(len(lens), bool)
    np.logical_or.at(has_inf, np.repeat(np.arange(len(lens)), lens), flat < 0)
    keep = ~has_inf & ((rp[:, 0] < n) | (rp[:, 1] < n))
    # polygon areas: fan of triangles (centroid, v_k, v_k+1) over the cyclically ordered ridge vertices
    rid = np.repeat(np.arange(len(lens)), lens)
    V = vor.vertices[np.where(flat < 0, 0, flat)]
    c0 = np.add.reduceat(V, start, axis=0) / lens[:, None]
    nxt = np.arange(flat.size) + 1
    last = start + lens - 1
    nxt[last] = start
    tri = 0.5 * np.linalg.norm(np.cross(V - c0[rid], V[nxt] - c0[rid]), axis=1)
    A = np.add.reduceat(tri, start)
    keep &= A > 1e-8 * h * h     # drop sliver faces (qhull round-off): < 1e-8 of a lattice face
    rp, A = rp[keep], A[keep]
    a, b = rp[:, 0], rp[:, 1]
    interior = (a < n) & (b < n)
    lo, hi = np.minimum(a, b)[interior], np.maximum(a, b)[interior]
    Ai = A[interior]
    di = np.linalg.norm(P[lo] - P[hi], axis=1)
    inner = np.where(a < n, a, b)[~interior]
    outer = np.where(a < n, b, a)[~interior]
    Ab = A[~interior]
    db = np.linalg.norm(P[inner] - allp[outer], axis=1) / 2.0
    if np.any(owner[outer - n] != inner):
        raise RuntimeError("a boundary ridge joins a point to another point's mirror")
    side = mface[outer - n]
    ax = side // 2
    vol = np.zeros(n)
    np.add.at(vol, lo, Ai * di / 6.0)
    np.add.at(vol, hi, Ai * di / 6.0)
    np.add.at(vol, inner, Ab * db / 3.0)
    fc = np.concatenate([np.stack([lo, hi], 1), np.stack([inner, np.full(inner.size, -1)], 1)]).astype(np.int32)
    ht = np.concatenate([np.stack([Ai * K[lo] / (di / 2), Ai * K[hi] / (di / 2)], 1),
                         np.stack([Ab * K[inner] / db, np.zeros(inner.size)], 1)])
    bc = np.concatenate([np.full(lo.size, BC_INTERIOR), np.where(ax == 0, BC_DIRICHLET, BC_NEUMANN)]).astype(np.uint8)
    area = np.concatenate([Ai, Ab])
    tie = np.concatenate([np.zeros(lo.size, np.int64), side])          # which cube face, for a cell's boundary faces
    order = np.lexsort((tie, fc[:, 1], fc[:, 0], bc != BC_INTERIOR))
    mesh = Mesh(n_cells=n, cell_volume=vol, face_cells=fc[order], half_trans=ht[order], face_bc=bc[order],
                face_area=area[order], shape=(n,), perm=K)
    mesh.points = P
    return mesh


def gaussian_random_field(shape, corr_cells, rng):
    """Zero-mean, unit-variance field with a Gaussian covariance of correlation length corr_cells (in cells).

    White noise on a grid padded to twice the size is filtered in Fourier space by the square root of the
    Gaussian spectral density, then cropped and standardised.
    """
    pad = tuple(2 * s for s in shape)
    noise = rng.standard_normal(pad)
    ks = np.meshgrid(*[np.fft.fftfreq(n) * 2 * np.pi for n in pad], indexing="ij")
    k2 = sum(k * k for k in ks)
    filt = np.exp(-0.25 * k2 * corr_cells ** 2)
    field_ = np.real(np.fft.ifftn(np.fft.fftn(noise) * filt))
    field_ = field_[tuple(slice(0, s) for s in shape)]
    field_ = (field_ - field_.mean()) / field_.std()
    return field_


def _to_lex(arr):
    """[nx, ny(, nz)] array -> lexicographic [N] vector with x fastest."""
    return np.asarray(arr).reshape(-1, order="F")


def lognormal_field(shape, sigma, corr_cells, seed):
    """K_0 = exp(sigma * g), g a standardised Gaussian random field."""
    rng = np.random.default_rng(seed)
    return _to_lex(np.exp(sigma * gaussian_random_field(shape, corr_cells, rng)))


def channelized_field(shape, decades, n_channels, seed, corr_cells=4.0):
    """log10 K_0 = GRF background + sinuous Gaussian channels (+3 decades) in horizontal layers, then rescaled
    affinely so that log10 K_0 spans [-decades/2, decades/2]."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = shape
    logk = gaussian_random_field(shape, corr_cells, rng)
    x = np.arange(nx)[:, None, None] + 0.5
    y = np.arange(ny)[None, :, None] + 0.5
    z = np.arange(nz)[None, None, :] + 0.5
    for _ in range(n_channels):
        width = rng.uniform(2.0, 4.0)
        z0 = rng.uniform(0, nz)
        y0 = rng.uniform(0, ny)
        amp = rng.uniform(0.1, 0.3) * ny
        lam = rng.uniform(0.5, 1.5) * nx
        phase = rng.uniform(0, 2 * np.pi)
        yc = y0 + amp * np.sin(2 * np.pi * x / lam + phase)
        dist2 = (y - yc) ** 2 + (z - z0) ** 2
        logk = logk + 3.0 * np.exp(-dist2 / (2.0 * (width / 2.0) ** 2))
    lo, hi = logk.min(), logk.max()
    logk = (logk - lo) / (hi - lo) * decades - decades / 2.0
    return _to_lex(10.0 ** logk)


@dataclass
class Problem:
    """A mesh plus nonlinearity, data and hierarchy options: one solve request."""
    mesh: Mesh
    kappa_kind: int
    kappa_a: float
    f_cell: np.ndarray               # [N] source density f|_K
    g_face: np.ndarray               # [F] Dirichlet value or Neumann flux density
    opts: dict = field(default_factory=dict)
    name: str = ""
    kappa_b: float = 0.0                    # second parameter (beta of the Richards kind)
    cell_shift: np.ndarray | None = None    # [N] cell heights z of the Richards kind (kappa depends on p - z)


def default_options(**kw):
    """Hierarchy and smoother options; the backtracking constants are the paper's (n_max = 4, theta = 0.9)."""
    o = dict(n_levels=2, agg_size=[16, 8, 8, 8, 8, 8, 8], modes=[2, 2, 2, 2, 2, 2, 2], nu_pre=2, nu_post=2,
             omega=0.8, bt_nmax=4, bt_theta=0.9, dp_clamp=0.0, coarsest_steps=10, tol_rel=1e-8, tol_abs=1e-10,
             max_cycles=50)
    o.update(kw)
    return o


def _dirichlet_data(mesh, g_left, g_right):
    g = np.zeros(mesh.n_faces)
    dir_faces = np.where(mesh.face_bc == BC_DIRICHLET)[0]
    # x-coordinate of the owning cell decides left/right
    nx = mesh.shape[0]
    i = mesh.face_cells[dir_faces, 0] % nx
    g[dir_faces] = np.where(i == 0, g_left, g_right)
    return g


def problem_config(name, scale=None):
    """Problems named by the workloads they stand in for.

    cart2d_32: 32x32 quadrilaterals, ln K ~ GRF(0,1) with correlation length 4 cells, kappa = exp(0.5 p),
      p = 1 left / 0 right, f = 0, aggregates of about 16 cells, 2 modes, 2 levels.
    chan3d_64: 64^3 hexahedra, channelized K over 6 decades, kappa = exp(2 p), aggregates of about 64 then 8
      cells, 4 modes, 3 levels. `scale` replaces 64 by a smaller side for tests.
    chan3d_256: 256^3 hexahedra (16.8M cells), channelized K over 8 decades (seed 5), kappa = exp(2 p), 5 levels
      (aggregates of about 64, then 8, 8, 8 cells), 6 modes per aggregate; its right-hand sides come from
      multi_rhs_rows. `scale` replaces 256 for smaller instances.
    """
    if name == "cart2d_32":
        n = scale or 32
        K = lognormal_field((n, n), 1.0, 4.0, seed=1)
        mesh = cartesian_mesh((n, n), K)
        g = _dirichlet_data(mesh, 1.0, 0.0)
        opts = default_options(n_levels=2, agg_size=[16, 8, 8, 8], modes=[2, 2, 2, 2])
        return Problem(mesh, KAPPA_EXP, 0.5, np.zeros(mesh.n_cells), g, opts, name)
    if name == "chan3d_64":
        n = scale or 64
        K = channelized_field((n, n, n), 6.0, 12, seed=2)
        mesh = cartesian_mesh((n, n, n), K)
        g = _dirichlet_data(mesh, 1.0, 0.0)
        opts = default_options(n_levels=3, agg_size=[64, 8, 8, 8], modes=[4, 4, 4, 4],
                               dp_clamp=float(np.log(1.5) / 2.0))
        return Problem(mesh, KAPPA_EXP, 2.0, np.zeros(mesh.n_cells), g, opts, name)
    if name == "chan3d_256":
        n = scale or 256
        K = channelized_field((n, n, n), 8.0, 12, seed=5)
        mesh = cartesian_mesh((n, n, n), K)
        g = _dirichlet_data(mesh, 1.0, 0.0)
        opts = default_options(n_levels=5, agg_size=[64, 8, 8, 8], modes=[6, 6, 6, 6],
                               dp_clamp=float(np.log(1.5) / 2.0))
        return Problem(mesh, KAPPA_EXP, 2.0, np.zeros(mesh.n_cells), g, opts, name)
    raise KeyError(name)


def voronoi_problem(n_side=12, seed=3):
    """Unstructured workload: clipped Voronoi cells of a jittered lattice, ln K_0 ~ N(0, 2^2) correlated over 4
    lattice spacings (sampled at the points), kappa = (1 + p^2)^-1, p = 1 on x = 0 and 0 on x = 1; pressure-change
    clamp 0.5 (half the range of the boundary data)."""
    field_ = gaussian_random_field((n_side,) * 3, 4.0, np.random.default_rng(seed + 100))

    def K_of(P):
        idx = np.clip((P * n_side).astype(int), 0, n_side - 1)
        return np.exp(2.0 * field_[idx[:, 0], idx[:, 1], idx[:, 2]])

    mesh = voronoi_mesh(n_side, K_of, seed=seed)
    g = np.zeros(mesh.n_faces)
    d = np.where(mesh.face_bc == BC_DIRICHLET)[0]
    g[d] = np.where(mesh.points[mesh.face_cells[d, 0], 0] < 0.5, 1.0, 0.0)
    opts = default_options(n_levels=3, agg_size=[27, 8, 8], modes=[4, 3, 3], dp_clamp=0.5)
    return Problem(mesh, KAPPA_INV1P2, 0.0, np.zeros(mesh.n_cells), g, opts, "voronoi")


def multi_rhs_rows(mesh, n_rhs, seed):
    """n_rhs data sets on one Cartesian mesh: per row a Dirichlet value U[0.5, 1.5] on x = 0 and U[-0.5, 0.5] on
    x = 1, and a smooth source density, the sum of 4 seeded Gaussian bumps (centres U[0.2, 0.8]^d, amplitudes
    U[-0.5, 0.5], width^2 = 0.01 of the unit box). Returns F [n_rhs, N] and G [n_rhs, F]."""
    rng = np.random.default_rng(seed)
    shape = mesh.shape
    d = np.where(mesh.face_bc == BC_DIRICHLET)[0]
    left = mesh.face_cells[d, 0] % shape[0] == 0
    x = (np.stack(np.unravel_index(np.arange(mesh.n_cells), shape, order="F"), axis=1) + 0.5) / np.array(shape)
    F = np.zeros((n_rhs, mesh.n_cells))
    G = np.zeros((n_rhs, mesh.n_faces))
    for r in range(n_rhs):
        G[r, d] = np.where(left, rng.uniform(0.5, 1.5), rng.uniform(-0.5, 0.5))
        for _ in range(4):
            c = rng.uniform(0.2, 0.8, len(shape))
            F[r] += rng.uniform(-0.5, 0.5) * np.exp(-np.sum((x - c) ** 2, axis=1) / 0.02)
    return F, G


CONFIGS = ("cart2d_32", "chan3d_64")


# alpha, beta and k0 [cm/day] of the two media of the Richards example (Sec. 4.3, Table richard-parameters)
RICHARDS_MEDIA = {"loam": (1.246e2, 1.77, 1.067e0), "sand": (1.175e6, 4.74, 8.160e2)}


def richards_problem(medium="loam", refine=0):
    """Static Richards' equation (Sec. 4.3, Example 3) on (0, 4000) x (0, 1000) (lengths in cm, the units of the
    media's parameters), 160 x 40 cells refined `refine` times by 2 in each direction; K_0 = k0 of the medium,
    kappa_K(p) = alpha / (alpha + |p - z_K|^beta) with p = psi + z and z_K the cell centre's height; f = 0.
    The paper gives the boundary conditions only in a figure; assumed here: no flow through the sides, the water
    table at the bottom (psi = 0, p = 0 on z = 0), and on the top (z = 1000) a ponded strip psi = 0 (p = 1000) on
    x < 1000 and a dry surface psi = -500 (p = 500) elsewhere. FAS options: aggregates of 36 cells on every level
    (the example's coarsening factor), 3 levels on the 160 x 40 mesh and 4 on refined ones, 4 spectral modes, at most
    4 halvings in Algorithm 1 for loam and 10 for sand (as in the example), no pressure-change clamp."""
    alpha, beta, k0 = RICHARDS_MEDIA[medium]
    nx, nz = 160 * 2 ** refine, 40 * 2 ** refine
    Lx, Lz = 4000.0, 1000.0
    mesh = cartesian_mesh((nx, nz), np.full(nx * nz, k0), lengths=(Lx, Lz), dirichlet_axes=(1,))
    hx, hz = Lx / nx, Lz / nz
    z_cell = (np.arange(nx * nz) // nx + 0.5) * hz
    g = np.zeros(mesh.n_faces)
    dirf = np.where(mesh.face_bc == BC_DIRICHLET)[0]
    K = mesh.face_cells[dirf, 0]
    top = K // nx == nz - 1
    x_c = (K % nx + 0.5) * hx
    g[dirf] = np.where(top, np.where(x_c < 1000.0, Lz, Lz - 500.0), 0.0)
    levels = 3 if refine == 0 else 4
    opts = default_options(n_levels=levels, agg_size=[36] * 7, modes=[4] * 7,
                           bt_nmax=4 if medium == "loam" else 10)
    return Problem(mesh, KAPPA_RICHARDS, alpha, np.zeros(mesh.n_cells), g, opts, "richards_" + medium,
                   kappa_b=beta, cell_shift=z_cell)
