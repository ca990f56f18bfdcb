"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds no arithmetic of the solver.  It describes the workloads
(structured boxes and channels, their level hierarchy and boundary faces), the
sizes of the C-ABI vector layout, and seeded random fields: the linearisation
velocity w sampled at the Q2 nodes and a reference solution x*.

C-ABI vector layout (the paper's X_n of Eq. (3.2), Sec. 3): time-node blocks
a = 0..k; inside block a first the R velocity values (Q2 nodes numbered
lexicographically with x fastest, components interleaved: node*d + c), then the
S pressure values (cells numbered lexicographically with x fastest, d+1
P1disc coefficients per cell: cell*(d+1) + m).
"""
from __future__ import annotations

import dataclasses
import numpy as np

BASE_SEED = 2210

# Face bits of the Dirichlet mask: face f = 2*dir + side (side 0 = low, 1 = high).
FACE_XLO, FACE_XHI, FACE_YLO, FACE_YHI, FACE_ZLO, FACE_ZHI = (1 << i for i in range(6))


@dataclasses.dataclass(frozen=True)
class MeshSpec:
    """Structured mesh hierarchy: finest cells n, coarsened by 2 per level."""

    dim: int
    n: tuple            # finest-level cells per direction
    lo: tuple           # domain lower corner
    hi: tuple           # domain upper corner
    n_levels: int       # levels 0 (coarsest) .. n_levels-1 (finest)
    dirichlet: int      # bit mask of Dirichlet faces; the other faces are do-nothing
    # 2D only: cells removed from the domain, the box [x0, x1) x [y0, y1) of coarsest-level cell
    # indices (empty: none); its faces carry Dirichlet data (no-slip for the obstacle channel)
    obstacle: tuple = ()
    # velocity order r of the pair (Q_r)^d x P_{r-1}^disc: 2 (the default) or 4 (2D)
    order: int = 2

    def cells(self, level: int) -> tuple:
        f = 2 ** (self.n_levels - 1 - level)
        for ni in self.n:
            if ni % f:
                raise ValueError(f"cells {self.n} not divisible by 2^{self.n_levels - 1}")
        return tuple(ni // f for ni in self.n)

    def pure_dirichlet(self) -> bool:
        return self.dirichlet == (1 << (2 * self.dim)) - 1

    def obstacle_cells(self, level: int) -> tuple:
        """The obstacle box in the cell indices of `level`, (x0, x1, y0, y1), or ()."""
        if not self.obstacle:
            return ()
        f = 2 ** level
        return tuple(int(v) * f for v in self.obstacle)


def n_nodes(cells: tuple, order: int = 2) -> int:
    return int(np.prod([order * c + 1 for c in cells]))


def n_cells(cells: tuple) -> int:
    return int(np.prod(cells))


def pressure_dofs(dim: int, order: int = 2) -> int:
    """dim P_{order-1}: the pressure coefficients of one cell (d + 1 for order 2)."""
    from math import comb
    return comb(order - 1 + dim, dim)


def block_sizes(dim: int, cells: tuple, order: int = 2) -> tuple:
    """(R, S) of one time-node block: Q_r velocity and P_{r-1}disc pressure counts."""
    return dim * n_nodes(cells, order), pressure_dofs(dim, order) * n_cells(cells)


def n_dofs(dim: int, cells: tuple, k: int, order: int = 2) -> int:
    r, s = block_sizes(dim, cells, order)
    return (k + 1) * (r + s)


def node_coords(spec: MeshSpec, level: int) -> np.ndarray:
    """Coordinates of the Q2 nodes of one level, shape (n_nodes, dim), x fastest."""
    cells = spec.cells(level)
    axes = [np.linspace(spec.lo[i], spec.hi[i], spec.order * cells[i] + 1) for i in range(spec.dim)]
    grids = np.meshgrid(*axes, indexing="ij")
    # ravel in Fortran order so that x is the fastest index
    return np.stack([g.ravel(order="F") for g in grids], axis=1)


def _unit(spec: MeshSpec, xyz: np.ndarray) -> np.ndarray:
    lo = np.asarray(spec.lo, float)
    hi = np.asarray(spec.hi, float)
    return (xyz - lo) / (hi - lo)


def _sine_series_grad(rng, u: np.ndarray, dim: int, modes: int, scale: np.ndarray):
    """Gradient of psi = sum a_m prod_i sin(m_i pi u_i), a_m ~ N(0,1); u in [0,1]^dim."""
    idx = np.stack(np.meshgrid(*([np.arange(1, modes + 1)] * dim), indexing="ij"), -1).reshape(-1, dim)
    a = rng.standard_normal(len(idx))
    grad = np.zeros((u.shape[0], dim))
    for coef, m in zip(a, idx):
        s = np.sin(np.pi * m * u)
        c = np.cos(np.pi * m * u)
        for e in range(dim):
            term = coef * np.pi * m[e] * c[:, e] / scale[e]
            for i in range(dim):
                if i != e:
                    term = term * s[:, i]
            grad[:, e] += term
    return grad


def _repeat_nodes(wn: np.ndarray, k: int) -> np.ndarray:
    return np.repeat(wn.reshape(1, -1), k + 1, axis=0)


def fourier_w(spec: MeshSpec, k: int, seed: int = BASE_SEED, modes: int = 4, amp: float = 1.0,
              level: int | None = None) -> np.ndarray:
    """Divergence-free w = curl(stream function) at the Q2 nodes, max nodal |w| = amp.

    2D: psi = sum_{m,n<=modes} a_mn sin(m pi x) sin(n pi y), w = (psi_y, -psi_x).
    3D: w = curl(A1, A2, A3), each A_i such a series in three variables.
    Constant over the k+1 Radau nodes; returned as (k+1, R) in the C-ABI order.
    """
    level = spec.n_levels - 1 if level is None else level
    rng = np.random.default_rng(seed)
    xyz = node_coords(spec, level)
    u = _unit(spec, xyz)
    scale = np.asarray(spec.hi, float) - np.asarray(spec.lo, float)
    if spec.dim == 2:
        g = _sine_series_grad(rng, u, 2, modes, scale)
        w = np.stack([g[:, 1], -g[:, 0]], axis=1)
    else:
        gs = [_sine_series_grad(rng, u, 3, modes, scale) for _ in range(3)]
        # curl A = (dA3/dy - dA2/dz, dA1/dz - dA3/dx, dA2/dx - dA1/dy)
        w = np.stack([gs[2][:, 1] - gs[1][:, 2], gs[0][:, 2] - gs[2][:, 0], gs[1][:, 0] - gs[0][:, 1]], axis=1)
    w *= amp / max(np.max(np.linalg.norm(w, axis=1)), 1e-300)
    return _repeat_nodes(w, k)


def channel_w(spec: MeshSpec, k: int, seed: int = BASE_SEED, u_max: float = 1.5, pert: float = 0.3,
              level: int | None = None) -> np.ndarray:
    """Poiseuille profile u = 4 u_max y (H - y) / H^2 plus a seeded curl perturbation (max |pert|)."""
    level = spec.n_levels - 1 if level is None else level
    xyz = node_coords(spec, level)
    height = spec.hi[1] - spec.lo[1]
    y = xyz[:, 1] - spec.lo[1]
    base = np.zeros_like(xyz)
    base[:, 0] = 4.0 * u_max * y * (height - y) / height ** 2
    p = fourier_w(spec, 0, seed=seed, amp=pert, level=level)[0].reshape(-1, spec.dim)
    return _repeat_nodes(base + p, k)


def split_blocks(x: np.ndarray, dim: int, cells: tuple, k: int, order: int = 2):
    """Views (velocity (k+1, n_nodes, dim), pressure (k+1, n_cells, dim P)) of a C-ABI vector."""
    r, s = block_sizes(dim, cells, order)
    xb = x.reshape(k + 1, r + s)
    return xb[:, :r].reshape(k + 1, -1, dim), xb[:, r:].reshape(k + 1, -1, pressure_dofs(dim, order))


def reference_solution(spec: MeshSpec, k: int, seed: int = BASE_SEED + 1, level: int | None = None) -> np.ndarray:
    """x* ~ N(0,1) per DoF; with Dirichlet data on the whole boundary the mean of the
    cell-constant pressure coefficients is removed per time node (zero pressure mean)."""
    level = spec.n_levels - 1 if level is None else level
    cells = spec.cells(level)
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(n_dofs(spec.dim, cells, k, spec.order))
    if spec.pure_dirichlet():
        _, p = split_blocks(x, spec.dim, cells, k, spec.order)
        p[:, :, 0] -= p[:, :, 0].mean(axis=1, keepdims=True)
    return x


def random_vector(n: int, seed: int) -> np.ndarray:
    return np.random.default_rng(seed).standard_normal(n)


# --- Workloads -----------------------------------------------------------------------------
ALL2 = (1 << 4) - 1
ALL3 = (1 << 6) - 1

WORKLOADS = {
    # 2D Oseen, unit square 8x8, levels 2x2..8x8, dG(0), tau=0.01, nu=1e-3, V(2,2), omega=0.7
    "square8_k0": dict(spec=MeshSpec(2, (8, 8), (0.0, 0.0), (1.0, 1.0), 3, ALL2), k=0, nu=1e-3,
                       tau=0.01, newton=False, w="fourier", nu1=2, nu2=2),
    # 2D channel [0,2.2]x[0,0.41], 704x128 -> 88x16, dG(1), tau=0.005, nu=1e-3, Newton Jacobian;
    # Dirichlet on inflow and walls, do-nothing outflow at x=2.2
    "channel704_k1": dict(spec=MeshSpec(2, (704, 128), (0.0, 0.0), (2.2, 0.41), 4,
                                        FACE_XLO | FACE_YLO | FACE_YHI), k=1, nu=1e-3, tau=0.005,
                          newton=True, w="channel", nu1=2, nu2=2),
    # 2D unit square 256x256 -> 16x16, k = 1..4
    "square256": dict(spec=MeshSpec(2, (256, 256), (0.0, 0.0), (1.0, 1.0), 5, ALL2), k=1, nu=1e-3,
                      tau=0.01, newton=False, w="fourier", nu1=2, nu2=2),
    # 3D unit cube 48^3 -> 6^3, dG(1)
    "cube48_k1": dict(spec=MeshSpec(3, (48, 48, 48), (0.0,) * 3, (1.0,) * 3, 4, ALL3), k=1, nu=1e-3,
                      tau=0.01, newton=False, w="fourier", nu1=2, nu2=2),
    # the paper's 2D element (Q4)^2 x P3disc on the channel, 352x64 quads -> 44x8 (4 levels): the
    # same Q_r node grid as the 704x128 Q2 channel
    "channel_q4": dict(spec=MeshSpec(2, (352, 64), (0.0, 0.0), (2.2, 0.41), 4, FACE_XLO | FACE_YLO | FACE_YHI,
                                     order=4), k=1, nu=1e-3, tau=0.005, newton=True, w="channel", nu1=2, nu2=2),
    # 3D unit cube 32^3 -> 4^3 for the robustness study in k = 0, 1, 2 (Sec. 4, Table 3.2)
    "cube32": dict(spec=MeshSpec(3, (32, 32, 32), (0.0,) * 3, (1.0,) * 3, 4, ALL3), k=1, nu=1e-3,
                   tau=0.01, newton=False, w="fourier", nu1=2, nu2=2),
}


def make_w(name_or_cfg, level: int | None = None, seed: int = BASE_SEED) -> np.ndarray:
    cfg = WORKLOADS[name_or_cfg] if isinstance(name_or_cfg, str) else name_or_cfg
    if cfg["w"] == "channel":
        return channel_w(cfg["spec"], cfg["k"], seed=seed, level=level)
    return fourier_w(cfg["spec"], cfg["k"], seed=seed, level=level)


def scaled(spec: MeshSpec, factor: int, n_levels: int | None = None) -> MeshSpec:
    """The same domain and faces with the finest cell counts divided by `factor`."""
    return dataclasses.replace(spec, n=tuple(c // factor for c in spec.n),
                               n_levels=spec.n_levels if n_levels is None else n_levels)


def smoothed_dofs_per_cycle(spec: MeshSpec, k: int, nu1: int, nu2: int) -> int:
    """Space-time DoFs smoothed by one V-cycle: sum over levels >= 1 of (nu1 + nu2) N_l."""
    return sum((nu1 + nu2) * n_dofs(spec.dim, spec.cells(l), k, spec.order) for l in range(1, spec.n_levels))



# ---------------------------------------------------------------- time march with a learned warm start
# 2D channel 128x32 -> 16x4, dG(1), tau=0.005, nu=1e-3, 400 slabs; the initial velocity is the
# Poiseuille profile plus a seeded curl perturbation of amplitude 0.5 (an impulsive start: the
# perturbation need not satisfy the boundary conditions); inflow data g = Poiseuille profile at
# every Radau node; the network is trained on slabs 1-200 and evaluated on 201-400.
MARCH = dict(spec=MeshSpec(2, (128, 32), (0.0, 0.0), (2.2, 0.41), 4, FACE_XLO | FACE_YLO | FACE_YHI), k=1,
             nu=1e-3, tau=0.005, slabs=400, train_slabs=200, pert=0.5, channels=(4, 16, 16, 4))


# ---------------------------------------------------------------- channel with an obstacle
# A structured stand-in for the benchmark of Sec. 4 (flow around an obstacle in a channel): the
# channel [0, 2.2] x [0, 0.41] with a square of cells removed around (0.2, 0.2), no-slip on its
# faces and on the walls, the Poiseuille profile at the inflow, do-nothing outflow.
OBSTACLE = dict(spec=MeshSpec(2, (176, 32), (0.0, 0.0), (2.2, 0.41), 3, FACE_XLO | FACE_YLO | FACE_YHI,
                              (3, 5, 3, 5)),
                k=1, nu=1e-3, tau=0.01, u_max=1.5, slabs=40)


def obstacle_node_mask(spec: MeshSpec, level: int | None = None) -> np.ndarray:
    """(n_nodes,) bool: Q2 nodes of the level that belong to a removed cell (on the obstacle's
    faces or inside it)."""
    level = spec.n_levels - 1 if level is None else level
    cells = spec.cells(level)
    nn = [2 * c + 1 for c in cells]
    out = np.zeros(nn[0] * nn[1], dtype=bool)
    box = spec.obstacle_cells(level)
    if not box:
        return out
    ix = np.arange(nn[0])
    iy = np.arange(nn[1])
    inx = (ix >= 2 * box[0]) & (ix <= 2 * box[1])
    iny = (iy >= 2 * box[2]) & (iy <= 2 * box[3])
    return (iny[:, None] & inx[None, :]).ravel()


def obstacle_inflow(spec: MeshSpec, k: int, u_max: float = 1.5) -> np.ndarray:
    """Dirichlet data (k+1, R): the Poiseuille profile, zero on the obstacle (no-slip)."""
    g = channel_w(spec, k, u_max=u_max, pert=0.0)
    g.reshape(k + 1, -1, spec.dim)[:, obstacle_node_mask(spec)] = 0.0
    return g


def march_initial_velocity(spec: MeshSpec, seed: int = BASE_SEED, pert: float = 0.5) -> np.ndarray:
    """v(0) at the finest Q2 nodes, (R,) in the C-ABI order."""
    return channel_w(spec, 0, seed=seed, pert=pert)[0].copy()


def march_inflow(spec: MeshSpec, k: int) -> np.ndarray:
    """Dirichlet data g: the Poiseuille profile (u_max = 1.5) at every Radau node, (k+1, R)."""
    return channel_w(spec, k, pert=0.0)


def cnn_init(channels, seed: int = BASE_SEED, last_scale: float = 0.1) -> np.ndarray:
    """Flat initial parameters of the warm-start network: per layer w[c_out][c_in][3][3] ~
    N(0, 1/(9 c_in)) (the last layer's scaled by last_scale), then zero biases; float32."""
    rng = np.random.default_rng(seed)
    out = []
    for li, (cin, cout) in enumerate(zip(channels[:-1], channels[1:])):
        w = rng.standard_normal(cout * cin * 9) / np.sqrt(9.0 * cin)
        if li == len(channels) - 2:
            w *= last_scale
        out += [w, np.zeros(cout)]
    return np.concatenate(out).astype(np.float32)


def batch_problems(count: int = 64, seed: int = BASE_SEED):
    """Uneven batch of 2D problems: n_x, n_y uniform in {32, 64, 128, 256}, k uniform in {1, 2},
    coarsened by 2 until min(n_x, n_y) = 4, Dirichlet on all faces, tau = 0.01, nu = 1e-3;
    problem i uses w and x* seeds BASE_SEED + i and BASE_SEED + i + 1 (as square8_k0).  The
    domain is [0, n_x / m] x [0, n_y / m] with m = max(n_x, n_y), so every cell is a square
    (on the unit square a 32 x 256 mesh has cells of aspect ratio 8, on which the Vanka
    V-cycle, in the oracle as on the GPU, stalls).  Returns [(spec, k, seed_i)]."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        nx, ny = (int(v) for v in rng.choice([32, 64, 128, 256], 2))
        k = int(rng.choice([1, 2]))
        levels = int(np.log2(min(nx, ny) // 4)) + 1
        m = max(nx, ny)
        out.append((MeshSpec(2, (nx, ny), (0.0, 0.0), (nx / m, ny / m), levels, ALL2), k, seed + i))
    return out
