"""Seeded synthetic problem generators (input synthesis only).

This module builds the sparse SPD matrices and right-hand sides that the
solver and its oracle are run on.  It holds none of the AMG method's
arithmetic: strength, coarsening, interpolation, Galerkin products, smoothing
and CG all live elsewhere.  Both the CUDA path and the CPU oracle take their
inputs from here, and nothing else is shared between them.

Workloads (all matrices CSR, int32 indices, float64 values, columns sorted
ascending within each row, Dirichlet boundary rows eliminated):

* ``poisson1d(n)``           tridiag(-1, 2, -1)
* ``poisson2d(N)``           5-point stencil 4/-1 on an N x N interior grid
* ``poisson3d(N)``           7-point stencil 6/-1 on an N^3 interior grid
* ``diffusion3d(N, sigma, seed)``  cell-centred 7-point heterogeneous diffusion
  whose face coefficient is the harmonic mean 2 k_i k_j / (k_i + k_j) of
  k = exp(g), g ~ N(0, sigma^2) i.i.d. smoothed by three passes of a 3x3x3 box
  mean truncated at the domain boundary; a domain-boundary face uses k_i, so
  k == 1 reproduces ``poisson3d`` exactly.
* ``graph_laplacian_spd(n, deg, shift, seed)``  random weighted graph
  Laplacian plus ``shift * I`` (unstructured SPD test matrices).

The paper's benchmark matrices (its Table 1) are not available; these
synthetic operators stand in for its fluid-dynamics (Laplace-type) class.
Grid ordering is lexicographic with x fastest: p = i + N*j + N*N*k.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class CSR:
    """A square sparse matrix in compressed-sparse-row form."""

    n: int
    rowptr: np.ndarray  # int32 [n+1]
    col: np.ndarray  # int32 [nnz]
    val: np.ndarray  # float64 [nnz]
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def to_dense(self) -> np.ndarray:
        d = np.zeros((self.n, self.n))
        rows = np.repeat(np.arange(self.n), np.diff(self.rowptr))
        d[rows, self.col] = self.val
        return d

    def matvec(self, x: np.ndarray) -> np.ndarray:
        """y = A x in float64 (used only to synthesise b = A x*)."""
        prod = self.val * x[self.col]
        rows = np.repeat(np.arange(self.n), np.diff(self.rowptr))
        return np.bincount(rows, weights=prod, minlength=self.n)


def _finish(n: int, cols: np.ndarray, vals: np.ndarray, mask: np.ndarray, meta=None) -> CSR:
    """Compress a dense (n, w) candidate table into CSR, keeping row-major order."""
    counts = mask.sum(axis=1, dtype=np.int64)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    if rowptr[-1] >= 2**31:
        raise ValueError("nnz does not fit int32")
    col = cols[mask].astype(np.int32, copy=False)
    val = vals[mask].astype(np.float64, copy=False)
    return CSR(n, rowptr.astype(np.int32), np.ascontiguousarray(col), np.ascontiguousarray(val), meta or {})


def poisson1d(n: int) -> CSR:
    i = np.arange(n, dtype=np.int64)
    cols = np.stack([i - 1, i, i + 1], axis=1)
    vals = np.tile(np.array([-1.0, 2.0, -1.0]), (n, 1))
    mask = (cols >= 0) & (cols < n)
    return _finish(n, cols, vals, mask, {"kind": "poisson1d"})


def poisson2d(N: int) -> CSR:
    n = N * N
    p = np.arange(n, dtype=np.int64)
    ix, iy = p % N, p // N
    cols = np.stack([p - N, p - 1, p, p + 1, p + N], axis=1)
    vals = np.tile(np.array([-1.0, -1.0, 4.0, -1.0, -1.0]), (n, 1))
    mask = np.stack([iy > 0, ix > 0, np.ones(n, bool), ix < N - 1, iy < N - 1], axis=1)
    return _finish(n, cols, vals, mask, {"kind": "poisson2d", "N": N})


def _box_mean_truncated(g: np.ndarray, passes: int) -> np.ndarray:
    """Three-axis 3-point mean truncated at the boundary, applied ``passes`` times.

    The truncated 3x3x3 box mean over in-bounds cells equals the composition
    of the truncated 1-D means along each axis, because the in-bounds part of
    the box is a product of intervals.
    """
    for _ in range(passes):
        for ax in range(3):
            s = g.copy()
            cnt = np.ones(g.shape[ax])
            lo = [slice(None)] * 3
            hi = [slice(None)] * 3
            lo[ax], hi[ax] = slice(1, None), slice(None, -1)
            s[tuple(lo)] += g[tuple(hi)]
            s[tuple(hi)] += g[tuple(lo)]
            cnt[1:] += 1
            cnt[:-1] += 1
            shape = [1, 1, 1]
            shape[ax] = -1
            g = s / cnt.reshape(shape)
    return g


def _stencil7(N: int, kx_m, kx_p, ky_m, ky_p, kz_m, kz_p, diag, meta) -> CSR:
    """Assemble a 7-point operator from per-cell face coefficients (arrays of n)."""
    n = N ** 3
    p = np.arange(n, dtype=np.int64)
    ix, iy, iz = p % N, (p // N) % N, p // (N * N)
    cols = np.stack([p - N * N, p - N, p - 1, p, p + 1, p + N, p + N * N], axis=1)
    vals = np.stack([-kz_m, -ky_m, -kx_m, diag, -kx_p, -ky_p, -kz_p], axis=1)
    mask = np.stack([iz > 0, iy > 0, ix > 0, np.ones(n, bool), ix < N - 1, iy < N - 1, iz < N - 1], axis=1)
    return _finish(n, cols, vals, mask, meta)


def poisson3d(N: int) -> CSR:
    n = N ** 3
    one = np.ones(n)
    return _stencil7(N, one, one, one, one, one, one, 6.0 * one, {"kind": "poisson3d", "N": N})


def diffusion_coefficients(N: int, sigma: float, rng: np.random.Generator) -> np.ndarray:
    """k = exp(g), g ~ N(0, sigma^2) i.i.d. then three truncated 3x3x3 box means.

    Returned as an (N, N, N) array indexed [z, y, x]."""
    g = rng.normal(0.0, sigma, size=N ** 3).reshape(N, N, N)
    g = _box_mean_truncated(g, passes=3)
    return np.exp(g)


def diffusion3d_from_k(k: np.ndarray, meta=None) -> CSR:
    """Cell-centred 7-point operator with harmonic-mean face coefficients."""
    N = k.shape[0]
    n = N ** 3

    def hm(a, b):
        return 2.0 * a * b / (a + b)

    kx_m = k.copy(); kx_m[:, :, 1:] = hm(k[:, :, 1:], k[:, :, :-1])
    kx_p = k.copy(); kx_p[:, :, :-1] = hm(k[:, :, :-1], k[:, :, 1:])
    ky_m = k.copy(); ky_m[:, 1:, :] = hm(k[:, 1:, :], k[:, :-1, :])
    ky_p = k.copy(); ky_p[:, :-1, :] = hm(k[:, :-1, :], k[:, 1:, :])
    kz_m = k.copy(); kz_m[1:, :, :] = hm(k[1:, :, :], k[:-1, :, :])
    kz_p = k.copy(); kz_p[:-1, :, :] = hm(k[:-1, :, :], k[1:, :, :])
    faces = [a.reshape(n) for a in (kx_m, kx_p, ky_m, ky_p, kz_m, kz_p)]
    diag = ((((faces[4] + faces[2]) + faces[0]) + faces[1]) + faces[3]) + faces[5]
    m = {"kind": "diffusion3d", "N": N, "k_min": float(k.min()), "k_max": float(k.max())}
    m.update(meta or {})
    return _stencil7(N, faces[0], faces[1], faces[2], faces[3], faces[4], faces[5], diag, m)


def diffusion3d(N: int, sigma: float, seed: int) -> tuple[CSR, np.random.Generator]:
    """Heterogeneous diffusion operator; returns (A, rng) with rng advanced past g."""
    rng = np.random.Generator(np.random.PCG64(seed))
    k = diffusion_coefficients(N, sigma, rng)
    return diffusion3d_from_k(k, {"sigma": sigma, "seed": seed}), rng


def graph_laplacian_spd(n: int, deg: int, shift: float, seed: int) -> CSR:
    """Random weighted graph Laplacian (weights in [0.5, 1.5]) plus shift * I."""
    rng = np.random.Generator(np.random.PCG64(seed))
    m = n * deg // 2
    a = rng.integers(0, n, size=m)
    b = rng.integers(0, n, size=m)
    keep = a != b
    a, b = a[keep], b[keep]
    w = rng.uniform(0.5, 1.5, size=a.size)
    d = np.zeros((n, n))
    np.add.at(d, (a, b), -w)
    np.add.at(d, (b, a), -w)
    np.fill_diagonal(d, 0.0)
    np.fill_diagonal(d, -d.sum(axis=1) + shift)
    return dense_to_csr(d, {"kind": "graph_laplacian", "seed": seed})


def graph_with_hubs(n: int, deg: int, hubs: int, hub_deg: int, shift: float, seed: int) -> CSR:
    """Random weighted graph Laplacian plus shift * I with a few high-degree hub
    nodes (long rows, wide Galerkin products)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    m = n * deg // 2
    a = list(rng.integers(0, n, size=m))
    b = list(rng.integers(0, n, size=m))
    for h in range(hubs):
        nb = rng.choice(n, size=hub_deg, replace=False)
        a += [h] * hub_deg
        b += list(nb)
    a, b = np.array(a), np.array(b)
    keep = a != b
    a, b = a[keep], b[keep]
    lo, hi = np.minimum(a, b), np.maximum(a, b)
    key = np.unique(lo.astype(np.int64) * n + hi)
    lo, hi = key // n, key % n
    w = rng.uniform(0.5, 1.5, size=lo.size)
    rows = np.concatenate([lo, hi, np.arange(n)])
    cols = np.concatenate([hi, lo, np.arange(n)])
    deg_w = np.bincount(lo, weights=w, minlength=n) + np.bincount(hi, weights=w, minlength=n)
    vals = np.concatenate([-w, -w, deg_w + shift])
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=rowptr[1:])
    return CSR(n, rowptr.astype(np.int32), cols.astype(np.int32), vals.astype(np.float64),
               {"kind": "graph_with_hubs", "seed": seed})


def dense_to_csr(d: np.ndarray, meta=None) -> CSR:
    n = d.shape[0]
    mask = d != 0.0
    np.fill_diagonal(mask, True)
    cols = np.broadcast_to(np.arange(n), (n, n))
    return _finish(n, cols, d, mask, meta)


def uniform(n: int, rng_or_seed) -> np.ndarray:
    rng = rng_or_seed if isinstance(rng_or_seed, np.random.Generator) else np.random.Generator(np.random.PCG64(rng_or_seed))
    return rng.uniform(-1.0, 1.0, size=n)


@dataclass
class Problem:
    name: str
    A: CSR
    b: np.ndarray
    xstar: np.ndarray | None


def config1() -> Problem:
    """2-D 5-point Poisson on 64 x 64, x* ~ U[-1,1] (seed 0), b = A x*."""
    A = poisson2d(64)
    xs = uniform(A.n, 0)
    return Problem("poisson2d_64", A, A.matvec(xs), xs)


def config2(N: int = 128) -> Problem:
    """3-D 7-point Poisson on N^3 (128^3 by default), x* ~ U[-1,1] (seed 1), b = A x*."""
    A = poisson3d(N)
    xs = uniform(A.n, 1)
    return Problem(f"poisson3d_{N}", A, A.matvec(xs), xs)


def config3(N: int = 256, sigma: float = 2.0, seed: int = 2) -> Problem:
    """Heterogeneous diffusion on N^3 (256^3 by default), b ~ U[-1,1] drawn after g."""
    A, rng = diffusion3d(N, sigma, seed)
    return Problem(f"diffusion3d_{N}", A, uniform(A.n, rng), None)


def nnz_poisson2d(N: int) -> int:
    """Closed form: 5n - 4N for the N x N interior 5-point stencil."""
    return 5 * N * N - 4 * N


def nnz_poisson3d(N: int) -> int:
    """Closed form: 7n - 6N^2 for the N^3 interior 7-point stencil."""
    return 7 * N ** 3 - 6 * N * N


def diffusion3d_device(N: int, sigma: float, seed: int, device="cuda", stream=None) -> CSR:
    """``diffusion3d``'s recipe generated on the GPU with torch (Philox normals from
    ``seed``), for request streams where host generation would dominate.  Same
    operator family (log-normal box-smoothed coefficients, harmonic-mean faces,
    7-point stencil, row order [z-, y-, x-, diag, x+, y+, z+]); a different random
    stream than the numpy version, so the matrices differ from ``diffusion3d``'s.
    Returns a CSR whose arrays are CUDA tensors (int32 / float64)."""
    import torch

    import contextlib

    ctx = torch.cuda.stream(stream) if stream is not None else contextlib.nullcontext()
    with ctx:
        gen = torch.Generator(device=device)
        gen.manual_seed(int(seed))
        g = torch.randn((N, N, N), generator=gen, device=device, dtype=torch.float64) * sigma
        for _ in range(3):
            for ax in range(3):
                s = g.clone()
                cnt = torch.ones(N, device=device, dtype=torch.float64)
                lo = [slice(None)] * 3
                hi = [slice(None)] * 3
                lo[ax], hi[ax] = slice(1, None), slice(None, -1)
                s[tuple(lo)] += g[tuple(hi)]
                s[tuple(hi)] += g[tuple(lo)]
                cnt[1:] += 1
                cnt[:-1] += 1
                shape = [1, 1, 1]
                shape[ax] = -1
                g = s / cnt.reshape(shape)
        k = torch.exp(g)

        def hm(a, b):
            return 2.0 * a * b / (a + b)

        kx_m = k.clone(); kx_m[:, :, 1:] = hm(k[:, :, 1:], k[:, :, :-1])
        kx_p = k.clone(); kx_p[:, :, :-1] = hm(k[:, :, :-1], k[:, :, 1:])
        ky_m = k.clone(); ky_m[:, 1:, :] = hm(k[:, 1:, :], k[:, :-1, :])
        ky_p = k.clone(); ky_p[:, :-1, :] = hm(k[:, :-1, :], k[:, 1:, :])
        kz_m = k.clone(); kz_m[1:, :, :] = hm(k[1:, :, :], k[:-1, :, :])
        kz_p = k.clone(); kz_p[:-1, :, :] = hm(k[:-1, :, :], k[1:, :, :])
        n = N ** 3
        f = [a.reshape(n) for a in (kx_m, kx_p, ky_m, ky_p, kz_m, kz_p)]
        diag = ((((f[4] + f[2]) + f[0]) + f[1]) + f[3]) + f[5]
        p = torch.arange(n, device=device, dtype=torch.int64)
        ix, iy, iz = p % N, (p // N) % N, p // (N * N)
        cols = torch.stack([p - N * N, p - N, p - 1, p, p + 1, p + N, p + N * N], dim=1)
        vals = torch.stack([-f[4], -f[2], -f[0], diag, -f[1], -f[3], -f[5]], dim=1)
        mask = torch.stack([iz > 0, iy > 0, ix > 0, torch.ones_like(ix, dtype=torch.bool), ix < N - 1, iy < N - 1,
                            iz < N - 1], dim=1)
        rowptr = torch.zeros(n + 1, device=device, dtype=torch.int64)
        torch.cumsum(mask.sum(dim=1), 0, out=rowptr[1:])
        col = cols[mask].to(torch.int32)
        val = vals[mask].contiguous()
        rp = rowptr.to(torch.int32)
    return CSR(n, rp, col, val, {"kind": "diffusion3d_device", "N": N, "sigma": sigma, "seed": seed})


def q1_hex_stiffness(nu: float) -> np.ndarray:
    """24 x 24 stiffness of the unit-cube trilinear (Q1) hexahedron for E = 1, by 2x2x2 Gauss
    quadrature.  Local node l = a + 2b + 4c sits at (a, b, c) in {0, 1}^3; dof 3l + comp."""
    lam = nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = 1.0 / (2.0 * (1.0 + nu))
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    D[np.arange(3), np.arange(3)] = lam + 2.0 * mu
    D[np.arange(3, 6), np.arange(3, 6)] = mu
    corners = np.array([[a, b, c] for c in (0, 1) for b in (0, 1) for a in (0, 1)], dtype=float)
    sgn = 2.0 * corners - 1.0  # reference coordinates of the corners in [-1, 1]^3
    gp = np.array([-1.0, 1.0]) / np.sqrt(3.0)
    K = np.zeros((24, 24))
    for xi in gp:
        for eta in gp:
            for zeta in gp:
                q = np.array([xi, eta, zeta])
                # dN_l/dxi_d = sgn_ld / 8 * prod_{e != d} (1 + sgn_le q_e); x = (xi + 1) / 2 so d/dx = 2 d/dxi
                dN = np.zeros((8, 3))
                for d in range(3):
                    o = [e for e in range(3) if e != d]
                    dN[:, d] = sgn[:, d] / 8.0 * (1 + sgn[:, o[0]] * q[o[0]]) * (1 + sgn[:, o[1]] * q[o[1]]) * 2.0
                B = np.zeros((6, 24))
                for l in range(8):
                    gx, gy, gz = dN[l]
                    B[0, 3 * l] = gx
                    B[1, 3 * l + 1] = gy
                    B[2, 3 * l + 2] = gz
                    B[3, 3 * l], B[3, 3 * l + 1] = gy, gx
                    B[4, 3 * l + 1], B[4, 3 * l + 2] = gz, gy
                    B[5, 3 * l], B[5, 3 * l + 2] = gz, gx
                K += B.T @ D @ B * (1.0 / 8.0)  # det(J) = 1/8, Gauss weights 1
    return 0.5 * (K + K.T)  # exactly symmetric


def elasticity3d(ne: int, nu: float = 0.3, layer: int = 8, E=(1.0, 1e3)) -> CSR:
    """Linear elasticity on an ne^3 grid of unit Q1 hexahedra, Young's modulus E[0] / E[1] in
    alternating element layers of thickness ``layer`` along z, the z = 0 face clamped (its nodes
    eliminated).  Unknowns are node-major (x, y, z displacement per node); nodes are
    lexicographic with x fastest over the (ne+1) x (ne+1) x ne free nodes.  Every coupled node
    pair stores its full 3x3 block (entries that vanish are kept as explicit zeros), so
    nnz = 9 * (3(ne+1) - 2)^2 * (3 ne - 2)."""
    Kr = q1_hex_stiffness(nu).reshape(8, 3, 8, 3)
    m = ne + 1  # nodes per x / y line
    nz = ne  # free node layers (k = 1 .. ne)
    nn = m * m * nz
    I = np.arange(nn, dtype=np.int64)
    ix, iy, iz = I % m, (I // m) % m, I // (m * m) + 1  # iz: global layer index 1..ne
    ez_layer = np.arange(ne) // layer
    Ee = np.where(ez_layer % 2 == 0, E[0], E[1])  # modulus of element layer ez
    offs = [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
    blocks = np.zeros((nn, 27, 3, 3))
    present = np.zeros((nn, 27), dtype=bool)
    for o, (dx, dy, dz) in enumerate(offs):
        jx, jy, jz = ix + dx, iy + dy, iz + dz
        present[:, o] = (jx >= 0) & (jx < m) & (jy >= 0) & (jy < m) & (jz >= 1) & (jz <= ne)
        for a in (0, 1):
            for b in (0, 1):
                for c in (0, 1):
                    # element with node I at local (a, b, c); J at local (a+dx, b+dy, c+dz)
                    la, lb, lc = a + dx, b + dy, c + dz
                    if not (0 <= la <= 1 and 0 <= lb <= 1 and 0 <= lc <= 1):
                        continue
                    ex, ey, ez = ix - a, iy - b, iz - c
                    ok = present[:, o] & (ex >= 0) & (ex < ne) & (ey >= 0) & (ey < ne) & (ez >= 0) & (ez < ne)
                    li, lj = a + 2 * b + 4 * c, la + 2 * lb + 4 * lc
                    w = np.where(ok, Ee[np.clip(ez, 0, ne - 1)], 0.0)
                    blocks[:, o] += w[:, None, None] * Kr[li, :, lj, :][None]
    J = I[:, None] + np.array([dx + m * dy + m * m * dz for dx, dy, dz in offs])[None, :]
    # exact symmetry: block (I, o) and the transpose of block (J, 26 - o) summed the same
    # contributions in different orders; replace both by their mean
    Jc = np.where(present, J, 0)
    mirror = blocks[Jc, 26 - np.arange(27)[None, :]].transpose(0, 1, 3, 2)
    blocks = np.where(present[:, :, None, None], 0.5 * (blocks + mirror), 0.0)
    n = 3 * nn
    # row (I, c): for each neighbour o (ascending J), dofs 3J + d
    cols = (3 * J[:, None, :, None] + np.arange(3)[None, None, None, :])  # (nn, 1, 27, 3)
    cols = np.broadcast_to(cols, (nn, 3, 27, 3)).reshape(n, 81)
    vals = blocks.transpose(0, 2, 1, 3).reshape(n, 81)  # [I, c, o, d]
    mask = np.broadcast_to(present[:, None, :, None], (nn, 3, 27, 3)).reshape(n, 81)
    return _finish(n, cols, vals, mask, {"kind": "elasticity3d", "ne": ne, "nu": nu, "layer": layer,
                                         "E": list(E)})


def nnz_elasticity3d(ne: int) -> int:
    """Closed form: 9 (3(ne+1) - 2)^2 (3 ne - 2) for ``elasticity3d``."""
    return 9 * (3 * (ne + 1) - 2) ** 2 * (3 * ne - 2)


def config4(ne: int = 64, k: int = 16) -> tuple[CSR, np.ndarray]:
    """Q1 elasticity on ne^3 elements (64^3 by default: 811,200 free dofs) with k right-hand
    sides (uniform[-1, 1] per dof, seed 3), returned as an n x k row-major block."""
    A = elasticity3d(ne)
    rng = np.random.Generator(np.random.PCG64(3))
    return A, rng.uniform(-1.0, 1.0, size=(A.n, k))


def kron_identity(A: CSR, bs: int, full_blocks: bool = True) -> CSR:
    """The operator A (x) I_bs in node-major order: unknown (I, c) = bs I + c couples to (J, c)
    with a_IJ.  With ``full_blocks`` every coupled node pair stores its whole bs x bs block
    (the off-component entries as explicit zeros), as block set-up requires."""
    n = A.n * bs
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    deg = np.diff(A.rowptr)
    w = (bs if full_blocks else 1)
    cols = np.zeros((n, int(deg.max()) * w), dtype=np.int64)
    vals = np.zeros_like(cols, dtype=np.float64)
    mask = np.zeros_like(cols, dtype=bool)
    pos = np.arange(A.nnz) - A.rowptr[rows]
    for c in range(bs):
        r = rows * bs + c
        if full_blocks:
            for d in range(bs):
                cols[r, pos * bs + d] = A.col * bs + d
                vals[r, pos * bs + d] = A.val if d == c else 0.0
                mask[r, pos * bs + d] = True
        else:
            cols[r, pos] = A.col * bs + c
            vals[r, pos] = A.val
            mask[r, pos] = True
    return _finish(n, cols, vals, mask, {"kind": "kron_identity", "bs": bs, "full_blocks": full_blocks})
