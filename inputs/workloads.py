"""Workload recipes (inputs only; no method arithmetic).

Every workload is a plain description consumed by both the CUDA library's
Python binding and the CPU oracle:

* ``dim``, ``n`` (nodes per axis), ``h`` (cm) for structured grids of 4-node
  bilinear quads (2D) or 8-node trilinear hexes (3D); node index
  ``x + nx*(y + ny*z)``, element index ``ex + (nx-1)*(ey + (ny-1)*ez)``.
* per-element longitudinal / transverse diffusivity (cm^2/ms) and a unit fibre
  direction (3 components; the z component is ignored in 2D).
* stimuli: node index lists with start time, duration, amplitude (model units
  per ms, added to dV/dt), period and count.

Units follow the paper's examples (Section 3): ms, cm, cm^2/ms, mV.  Seeds are
``2011047 + index`` of the configuration they stand for.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np

SEED_BASE = 2011047

# Mitchell-Schaeffer parameters of the plain 2D configuration:
# tau_in, tau_out, tau_open, tau_close (ms), v_gate (dimensionless).
MS_DEFAULT_PARAMS = (0.3, 6.0, 120.0, 150.0, 0.13)


@dataclasses.dataclass
class Stimulus:
    nodes: np.ndarray          # int64 node indices
    t_start: float             # ms
    duration: float            # ms
    amplitude: float           # added to dV/dt (model units per ms)
    period: float = 0.0        # ms (ignored when count == 1)
    count: int = 1


@dataclasses.dataclass
class Workload:
    name: str
    model: str                               # "ms" | "tp06" | "cubic"
    model_params: tuple
    t_end: float                             # ms simulated
    dt: float = 0.1                          # splitting step (ms)
    dt0: float = 0.01                        # smallest reaction sub-step (ms)
    v_threshold: Optional[float] = None      # activation threshold (model units)
    # structured grid
    dim: int = 0
    n: tuple = (1, 1, 1)
    h: float = 0.0
    # unstructured tetrahedral mesh
    xyz: Optional[np.ndarray] = None         # (n_nodes, 3) cm
    tets: Optional[np.ndarray] = None        # (n_tets, 4) int64
    # per element conductivity
    d_long: Optional[np.ndarray] = None
    d_trans: Optional[np.ndarray] = None
    fibre: Optional[np.ndarray] = None       # (n_elem, 3) unit vectors
    stimuli: List[Stimulus] = dataclasses.field(default_factory=list)
    meta: dict = dataclasses.field(default_factory=dict)
    # TP06 cell type per node (0 endo, 1 epi, 2 mid-myocardial); None: the
    # type in model_params at every node
    cell_type: Optional[np.ndarray] = None

    @property
    def n_nodes(self) -> int:
        if self.xyz is not None:
            return int(self.xyz.shape[0])
        nx, ny, nz = (tuple(self.n) + (1, 1, 1))[:3]
        return int(nx * ny * (nz if self.dim == 3 else 1))

    @property
    def n_elems(self) -> int:
        if self.tets is not None:
            return int(self.tets.shape[0])
        nx, ny, nz = (tuple(self.n) + (1, 1, 1))[:3]
        if self.dim == 2:
            return (nx - 1) * (ny - 1)
        return (nx - 1) * (ny - 1) * (nz - 1)


def grid_node_coords(dim: int, n, h: float) -> np.ndarray:
    """(n_nodes, 3) coordinates of a structured grid, x fastest."""
    nx, ny = n[0], n[1]
    nz = n[2] if dim == 3 else 1
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return np.stack([x.ravel() * h, y.ravel() * h, z.ravel() * h], axis=1).astype(np.float64)


def _elem_centres(dim: int, n, h: float) -> np.ndarray:
    nx, ny = n[0], n[1]
    nz = n[2] if dim == 3 else 2
    ez, ey, ex = np.meshgrid(np.arange(nz - 1), np.arange(ny - 1), np.arange(nx - 1), indexing="ij")
    c = np.stack([(ex.ravel() + 0.5) * h, (ey.ravel() + 0.5) * h, (ez.ravel() + 0.5) * h], axis=1)
    if dim == 2:
        c[:, 2] = 0.0
    return c


# Stimulus amplitude for the TP06 corner stimulus (mV/ms, added to dV/dt for
# 2 ms): twice the capture threshold (~13.3 mV/ms, found by bisection on a
# 21 x 21 x 11 slab with the same spacing), following the "twice diastolic
# threshold" protocol of Section 3.1.
TP06_CORNER_AMP = 27.0

# Mitchell-Schaeffer left-column stimulus of the plain 2D square.  The literal
# 0.1/ms for 1 ms does not capture on the 41 x 41 grid (the tissue sink drains
# it below threshold); the capture threshold is ~0.5214/ms, and twice it is used.
MS_SQUARE_AMP = 1.04


def ms_square_2d(n: int = 41, length: float = 1.0, D: float = 0.001, t_end: float = 100.0,
                 amp: float = MS_SQUARE_AMP, dt: float = 0.1) -> Workload:
    """Plain 2D isotropic square, Mitchell-Schaeffer, left-column stimulus.

    1 cm x 1 cm, n x n nodes of bilinear quads, D = 0.001 cm^2/ms, 1 ms
    stimulus on the x = 0 column (``MS_SQUARE_AMP``), 0.1 ms splitting step.
    """
    h = length / (n - 1)
    ne = (n - 1) * (n - 1)
    left = np.arange(n, dtype=np.int64) * n
    return Workload(
        name=f"ms_square_{n}x{n}", model="ms", model_params=MS_DEFAULT_PARAMS, t_end=t_end,
        dt=dt, v_threshold=0.5, dim=2, n=(n, n, 1), h=h,
        d_long=np.full(ne, D), d_trans=np.full(ne, D), fibre=np.tile([1.0, 0.0, 0.0], (ne, 1)),
        stimuli=[Stimulus(left, 0.0, 1.0, amp)],
    )


def tp06_slab_3d(nx: int = 101, ny: int = 101, nz: int = 26, h: float = 0.02,
                 d_long: float = 0.0012, d_trans: float = 0.0003, t_end: float = 500.0,
                 celltype: int = 0, corner: float = 0.1, stim_dur: float = 2.0,
                 amp: float = TP06_CORNER_AMP, dt: float = 0.1, transmural: bool = False) -> Workload:
    """3D anisotropic slab (2 x 2 x 0.5 cm at the default size) of trilinear hexes.

    Fibres lie in the x-y plane and rotate linearly through the wall: the
    element whose centre is at height z_c has angle
    theta = -60 deg + 120 deg * z_c / L_z, fibre = (cos theta, sin theta, 0).
    Corner stimulus: all nodes with x, y, z <= ``corner`` cm for ``stim_dur`` ms.
    ``transmural``: TP06 cell type per node by wall depth instead of
    ``celltype`` everywhere: the lower third of the node layers endocardial,
    the middle third mid-myocardial, the upper third epicardial.
    """
    n = (nx, ny, nz)
    c = _elem_centres(3, n, h)
    lz = (nz - 1) * h
    theta = np.deg2rad(-60.0 + 120.0 * c[:, 2] / lz)
    fib = np.stack([np.cos(theta), np.sin(theta), np.zeros_like(theta)], axis=1)
    ne = c.shape[0]
    xyz = grid_node_coords(3, n, h)
    eps = 1e-9
    corner_nodes = np.nonzero((xyz[:, 0] <= corner + eps) & (xyz[:, 1] <= corner + eps)
                              & (xyz[:, 2] <= corner + eps))[0].astype(np.int64)
    cell_type = None
    if transmural:
        layer = np.arange(nx * ny * nz) // (nx * ny)
        cell_type = np.where(3 * layer < nz, 0, np.where(3 * layer < 2 * nz, 2, 1)).astype(np.uint8)
    return Workload(
        name=f"tp06_slab_{nx}x{ny}x{nz}" + ("_transmural" if transmural else ""), model="tp06",
        model_params=(float(celltype),), t_end=t_end, dt=dt, v_threshold=-40.0, dim=3, n=n, h=h,
        d_long=np.full(ne, d_long), d_trans=np.full(ne, d_trans), fibre=fib,
        stimuli=[Stimulus(corner_nodes, 0.0, stim_dur, amp)], cell_type=cell_type,
    )


SHEET_COLUMN_THRESHOLD = 257.4   # TP06, 1 ms pulse on the X = 0 column, h = 100 um (bisection, oracle)


def aniso_sheet_2d(n: int = 501, length: float = 5.0, d0: float = 0.0017, rho: float = 0.25,
                   model: str = "tp06", t_end: float = 500.0, amp: float = 2.0 * SHEET_COLUMN_THRESHOLD,
                   dt: float = 0.1) -> Workload:
    """2D sheet shaped like the paper's Section 3.1 example.

    5 x 5 cm, h = 100 um (n = 501 nodes per side, 251 001 nodes), fibres along
    X, d0 = 0.0017 cm^2/ms longitudinal and rho * d0 transverse, 1 ms stimulus
    on the X = 0 column at twice its capture threshold (Section 3.1; the
    threshold of a single column at h = 100 um is 257 mV/ms, found by bisection
    with the oracle on a 0.2 cm sheet).  The cell model is a stand-in (the
    paper's O'Hara-Rudy model is not available).
    """
    h = length / (n - 1)
    ne = (n - 1) * (n - 1)
    left = np.arange(n, dtype=np.int64) * n
    params = MS_DEFAULT_PARAMS if model == "ms" else (1.0,)
    vth = 0.5 if model == "ms" else -40.0
    a = 0.1 if model == "ms" else amp
    return Workload(
        name=f"sheet_{model}_{n}x{n}", model=model, model_params=params, t_end=t_end, dt=dt,
        v_threshold=vth, dim=2, n=(n, n, 1), h=h,
        d_long=np.full(ne, d0), d_trans=np.full(ne, rho * d0),
        fibre=np.tile([1.0, 0.0, 0.0], (ne, 1)),
        stimuli=[Stimulus(left, 0.0, 1.0, a)],
    )


def cubic_strip_2d(length: float = 2.0, h: float = 0.005, D: float = 0.001,
                   a: float = 0.1, a_r: float = 1.0, t_end: float = 60.0, dt: float = 0.01,
                   stim_len: float = 0.1) -> Workload:
    """Two-row strip for the bistable (Nagumo) front-speed check.

    The cubic test model dv/dt = a_r v (1 - v)(v - a) with diffusion D has an
    exact travelling front of speed sqrt(a_r D / 2)(1 - 2a).
    """
    nx = int(round(length / h)) + 1
    n = (nx, 2, 1)
    ne = (nx - 1)
    xs = np.arange(nx) * h
    left = np.nonzero(xs <= stim_len + 1e-9)[0]
    nodes = np.concatenate([left, left + nx]).astype(np.int64)
    return Workload(
        name=f"cubic_strip_h{h}", model="cubic", model_params=(a_r, a), t_end=t_end, dt=dt,
        dt0=dt / 10.0, v_threshold=0.5, dim=2, n=n, h=h,
        d_long=np.full(ne, D), d_trans=np.full(ne, D), fibre=np.tile([1.0, 0.0, 0.0], (ne, 1)),
        stimuli=[Stimulus(nodes, 0.0, 2.0, 1.0)],
    )


def _kuhn_tets(nx: int, ny: int, nz: int) -> np.ndarray:
    """Split every cube of an nx x ny x nz node grid into 6 tetrahedra.

    All six share the main diagonal (corner 0 -> corner 7); the split is
    conforming across cube faces because every cube is split the same way.
    Corner c of a cube has offsets (c & 1, (c >> 1) & 1, (c >> 2) & 1).
    """
    ez, ey, ex = np.meshgrid(np.arange(nz - 1), np.arange(ny - 1), np.arange(nx - 1), indexing="ij")
    base = (ex + nx * (ey + ny * ez)).ravel().astype(np.int64)
    off = np.array([0, 1, nx, nx + 1, nx * ny, nx * ny + 1, nx * ny + nx, nx * ny + nx + 1],
                   dtype=np.int64)
    # paths from corner 0 to corner 7 through one axis step at a time
    paths = [(0, 1, 3, 7), (0, 1, 5, 7), (0, 2, 3, 7), (0, 2, 6, 7), (0, 4, 5, 7), (0, 4, 6, 7)]
    tets = np.concatenate([base[:, None] + off[list(p)][None, :] for p in paths], axis=0)
    return tets


# S2 time of the S1-S2 cross-field protocol on the tet slab (ms): the only
# time of a 10 ms grid (200 .. 350 ms) after which activity persisted at
# 1000 ms in the oracle's scan of a reduced slab with the same in-plane mesh
# (tests/golden/s1s2_scan_oracle.json): the S2 wave enters tissue recovering
# from S1 and re-enters, about every 250 ms.  Earlier S2 meets refractory
# tissue; later S2 excites the slab once.
S1S2_S2_TIME = 320.0


def tet_slab_3d(nx: int = 201, ny: int = 201, nz: int = 51, h: float = 0.02,
                jitter: float = 0.2, fibrosis: float = 0.3, scar_radius: float = 0.5,
                scar_scale: float = 0.1, d_long: float = 0.0012, d_trans: float = 0.0003,
                t_end: float = 1000.0, s2_time: float = S1S2_S2_TIME, amp: float = 60.0,
                seed_index: int = 2) -> Workload:
    """Seeded jittered tetrahedral slab with diffuse fibrosis and a central scar.

    4 x 4 x 1 cm at the default size (201 x 201 x 51 nodes, h = 0.02 cm, about
    2.06 M nodes).  Interior nodes move by U(-jitter h, +jitter h) per axis;
    boundary nodes stay on their faces.  Cubes are split into 6 tetrahedra.
    Each tet becomes non-conducting (D = 0) with probability ``fibrosis``; a
    cylinder of radius ``scar_radius`` through the thickness at the slab centre
    has D scaled by ``scar_scale``.  Fibres rotate through the wall as in the
    structured slab.  S1: nodes with x <= 0.1 cm at t = 0; S2: x <= L/4,
    y <= L/2 at ``s2_time`` (cross-field protocol, Section 3.2).
    """
    rng = np.random.default_rng(SEED_BASE + seed_index)
    xyz = grid_node_coords(3, (nx, ny, nz), h)
    ix = np.arange(nx * ny * nz) % nx
    iy = (np.arange(nx * ny * nz) // nx) % ny
    iz = np.arange(nx * ny * nz) // (nx * ny)
    for axis, idx, nmax in ((0, ix, nx), (1, iy, ny), (2, iz, nz)):
        move = (idx > 0) & (idx < nmax - 1)
        xyz[move, axis] += rng.uniform(-jitter * h, jitter * h, size=int(move.sum()))
    tets = _kuhn_tets(nx, ny, nz)
    ne = tets.shape[0]
    cent = xyz[tets].mean(axis=1)
    lz = (nz - 1) * h
    theta = np.deg2rad(-60.0 + 120.0 * cent[:, 2] / lz)
    fib = np.stack([np.cos(theta), np.sin(theta), np.zeros_like(theta)], axis=1)
    scale = np.ones(ne)
    scale[rng.random(ne) < fibrosis] = 0.0
    lx, ly = (nx - 1) * h, (ny - 1) * h
    in_scar = (cent[:, 0] - lx / 2) ** 2 + (cent[:, 1] - ly / 2) ** 2 <= scar_radius ** 2
    scale[in_scar] *= scar_scale
    eps = 1e-9
    s1 = np.nonzero(xyz[:, 0] <= 0.1 + eps)[0].astype(np.int64)
    s2 = np.nonzero((xyz[:, 0] <= lx / 4 + eps) & (xyz[:, 1] <= ly / 2 + eps))[0].astype(np.int64)
    return Workload(
        name=f"tet_slab_{nx}x{ny}x{nz}", model="tp06", model_params=(0.0,), t_end=t_end,
        v_threshold=-40.0, dim=3, xyz=xyz, tets=tets,
        d_long=d_long * scale, d_trans=d_trans * scale, fibre=fib,
        stimuli=[Stimulus(s1, 0.0, 2.0, amp), Stimulus(s2, s2_time, 2.0, amp)],
        meta={"grid": (nx, ny, nz), "h": h},
    )


def lognormal_field_2d(n: int, h: float, corr_len: float = 0.2, sigma_log: float = 0.3,
                       median: float = 0.001, seed_index: int = 3) -> np.ndarray:
    """Seeded log-normal nodal field on an n x n grid.

    A unit-variance stationary Gaussian field with squared-exponential
    covariance exp(-r^2 / (2 l^2)) is drawn by spectral filtering of white noise
    on a periodic box twice the grid size, then ``median * exp(sigma_log * g)``.
    """
    rng = np.random.default_rng(SEED_BASE + seed_index)
    m = 2 * n
    k = np.fft.fftfreq(m, d=h) * 2.0 * np.pi
    kx, ky = np.meshgrid(k, k, indexing="ij")
    spec = np.exp(-0.25 * corr_len ** 2 * (kx ** 2 + ky ** 2))   # sqrt of the SE spectrum
    noise = rng.standard_normal((m, m))
    g = np.real(np.fft.ifft2(np.fft.fft2(noise) * spec))[:n, :n]
    g = (g - g.mean()) / g.std()
    return (median * np.exp(sigma_log * g)).ravel()


def ms_adjoint_2d(n: int = 256, h: float = 0.025, t_end: float = 200.0, n_sensors: int = 64,
                  sample_dt: float = 1.0, seed_index: int = 3):
    """Adjoint workload: n x n MS tissue with a log-normal nodal D field.

    Returns (workload, nodal_D, sensors, sample_dt).  Element D is the mean of
    its 4 nodal values (done by the consumers, not here).  The left-column
    stimulus uses twice the square's amplitude (the field lowers D in places,
    which raises the capture threshold).
    """
    d_node = lognormal_field_2d(n, h, seed_index=seed_index)
    rng = np.random.default_rng(SEED_BASE + 10 + seed_index)
    sensors = np.sort(rng.choice(n * n, size=n_sensors, replace=False)).astype(np.int64)
    ne = (n - 1) * (n - 1)
    left = np.arange(n, dtype=np.int64) * n
    wl = Workload(
        name=f"ms_adjoint_{n}x{n}", model="ms", model_params=MS_DEFAULT_PARAMS, t_end=t_end,
        v_threshold=0.5, dim=2, n=(n, n, 1), h=h,
        d_long=np.zeros(ne), d_trans=np.zeros(ne), fibre=np.tile([1.0, 0.0, 0.0], (ne, 1)),
        stimuli=[Stimulus(left, 0.0, 1.0, 2.0 * MS_SQUARE_AMP)],
    )
    return wl, d_node, sensors, sample_dt


def batch_tissues(n_tissues: int = 512, side_min: int = 32, side_max: int = 256,
                  h: float = 0.025, t_end: float = 300.0, seed_index: int = 4) -> List[Workload]:
    """Uneven batch of square 2D tissues with per-tissue D, model and stimulus site.

    Side length ~ U{side_min..side_max} nodes, D ~ U(0.0005, 0.002) cm^2/ms
    isotropic, MS and TP06 alternating (50/50), stimulus: a 3 x 3 node patch at
    a seeded site, 2 ms.
    """
    rng = np.random.default_rng(SEED_BASE + seed_index)
    out = []
    for t in range(n_tissues):
        s = int(rng.integers(side_min, side_max + 1))
        D = float(rng.uniform(0.0005, 0.002))
        model = "ms" if t % 2 == 0 else "tp06"
        sx, sy = int(rng.integers(0, s - 3)), int(rng.integers(0, s - 3))
        patch = np.array([(sx + i) + s * (sy + j) for j in range(3) for i in range(3)], dtype=np.int64)
        ne = (s - 1) * (s - 1)
        params = MS_DEFAULT_PARAMS if model == "ms" else (0.0,)
        amp = 2.0 if model == "ms" else 2.0 * TP06_CORNER_AMP
        out.append(Workload(
            name=f"tissue{t}", model=model, model_params=params, t_end=t_end,
            v_threshold=0.5 if model == "ms" else -40.0, dim=2, n=(s, s, 1), h=h,
            d_long=np.full(ne, D), d_trans=np.full(ne, D), fibre=np.tile([1.0, 0.0, 0.0], (ne, 1)),
            stimuli=[Stimulus(patch, 0.0, 2.0, amp)],
        ))
    return out


__all__ = [
    "Stimulus", "Workload", "grid_node_coords", "ms_square_2d", "tp06_slab_3d", "aniso_sheet_2d",
    "cubic_strip_2d", "tet_slab_3d", "lognormal_field_2d", "ms_adjoint_2d", "batch_tissues",
    "MS_DEFAULT_PARAMS", "SEED_BASE",
]
