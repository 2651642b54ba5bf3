"""Seeded synthetic inputs for the windowed LBM-LES solver and its discrete adjoint.

This module builds the input arrays of a problem -- node classes, the design
field gamma (1 = solid), objective weights, the inlet velocity profile -- and
the scalar parameters that go with them.  It holds none of the method's
arithmetic (no equilibrium, collision, boundary rule or adjoint): the CUDA
library and the CPU oracle each receive the same arrays and compute
everything from them on their own.

The five workload shapes follow the paper's numerical examples: a cylinder
channel (Sec. 4.2), a cylinder wake (Sec. 4.3), a backward-facing step
(Sec. 4.1) and a U-bend duct (Sec. 4.4, extruded to 3D).  Every random draw
comes from ``numpy.random.default_rng(seed)``; smoothing is
``scipy.ndimage.gaussian_filter``.

Array layout everywhere: ``[z][y][x]`` (x fastest), flattened index
``i = x + nx * (y + ny * z)``.
"""
from __future__ import annotations

import dataclasses
from dataclasses import dataclass, field

import numpy as np
from scipy.ndimage import gaussian_filter

# Node classes (match enum lbm_node_class in include/lbmadj.h).
FLUID, WALL, INLET, OUTLET_P, OUTLET_ZG = 0, 1, 2, 3, 4
# Objective kinds (enum lbm_objective_kind).
OBJ_DISSIPATION, OBJ_VELOCITY_DEV, OBJ_PRESSURE, OBJ_DRAG = 0, 1, 2, 3
# Monitored quantity of the window criterion (enum lbm_monitor_kind).
MON_DRAG, MON_OBJECTIVE = 0, 1
# Checkpoint storage (enum lbm_ckpt_format).
CKPT_NATIVE, CKPT_FP16, CKPT_BF16, CKPT_MOMENT = 0, 1, 2, 3


@dataclass
class Case:
    """One problem instance: geometry, design, objective and window settings."""

    name: str
    lattice: int                    # 9 (D2Q9) or 19 (D3Q19)
    nx: int
    ny: int
    nz: int
    tau: float                      # molecular relaxation time
    cs_smag: float                  # Smagorinsky constant (filter width 1)
    node_class: np.ndarray          # uint8 [nz][ny][nx]
    gamma: np.ndarray               # float64 [nz][ny][nx], 1 = solid
    inlet_u: np.ndarray             # float64 [nz][ny], x-velocity on the x=0 face
    obj_weights: np.ndarray         # float64 [nz][ny][nx]
    obj_kind: int = OBJ_DISSIPATION
    obj_uref: tuple = (0.0, 0.0, 0.0)
    q_interp: float = 0.1           # interpolation parameter of g(phi)
    g_max: float = 0.5              # g at phi = 0 (the paper's 0.5)
    rho_out: float = 1.0            # outlet / reference density
    periodic: tuple = (0, 0, 0)
    monitor_kind: int = MON_DRAG
    monitor_u: float = 0.05         # reference velocity of the drag coefficient
    monitor_l: float = 1.0          # reference length of the drag coefficient
    window_len: int = 200
    sample_every: int = 1
    sample_from: int = 0            # first sampled step of a window (full-time runs: T - |W|)
    conv_tol: float = 1e-3
    ckpt_every: int = 200
    ckpt_format: int = CKPT_NATIVE
    max_windows: int = 10
    design_box: tuple = (0, 0, 0, 0, 0, 0)   # x0,x1,y0,y1,z0,z1 (half-open)
    obj_box: tuple = field(default=None)     # filled from obj_weights if None

    def __post_init__(self):
        self.node_class = np.ascontiguousarray(self.node_class, dtype=np.uint8)
        self.gamma = np.ascontiguousarray(self.gamma, dtype=np.float64)
        self.inlet_u = np.ascontiguousarray(self.inlet_u, dtype=np.float64)
        self.obj_weights = np.ascontiguousarray(self.obj_weights, dtype=np.float64)
        shp = (self.nz, self.ny, self.nx)
        assert self.node_class.shape == shp and self.gamma.shape == shp
        assert self.obj_weights.shape == shp and self.inlet_u.shape == (self.nz, self.ny)
        if self.obj_box is None:
            self.obj_box = nonzero_box(self.obj_weights)

    @property
    def n(self) -> int:
        return self.nx * self.ny * self.nz

    def replace(self, **kw) -> "Case":
        kw.setdefault("obj_box", None if "obj_weights" in kw else self.obj_box)
        return dataclasses.replace(self, **kw)


def nonzero_box(w: np.ndarray) -> tuple:
    """Smallest half-open box (x0,x1,y0,y1,z0,z1) holding every nonzero of w."""
    nz_idx = np.nonzero(w)
    if len(nz_idx[0]) == 0:
        return (0, 0, 0, 0, 0, 0)
    z, y, x = nz_idx
    return (int(x.min()), int(x.max()) + 1, int(y.min()), int(y.max()) + 1,
            int(z.min()), int(z.max()) + 1)


def tau_from_re(u: float, length: float, re: float) -> float:
    """Relaxation time for a Reynolds number Re = U L / nu (Sec. 4, lattice units)."""
    nu = u * length / re
    return 3.0 * nu + 0.5


def smooth_noise(shape, sigma: float, seed: int) -> np.ndarray:
    """Gaussian-filtered standard-normal noise, seeded."""
    rng = np.random.default_rng(seed)
    return gaussian_filter(rng.standard_normal(shape), sigma, mode="nearest")


def scaled_noise(shape, sigma, amplitude, seed):
    """Smooth noise scaled so that max |noise| == amplitude."""
    n = smooth_noise(shape, sigma, seed)
    return n * (amplitude / np.max(np.abs(n)))


def minmax_noise(shape, sigma, seed):
    """Smooth noise rescaled to the range [0, 1]."""
    n = smooth_noise(shape, sigma, seed)
    return (n - n.min()) / (n.max() - n.min())


def disk_mask(nx, ny, cx, cy, diameter):
    y, x = np.mgrid[0:ny, 0:nx]
    return (x - cx) ** 2 + (y - cy) ** 2 <= (diameter / 2.0) ** 2


def parabolic_profile(ny, u_max):
    """u(y) = 4 u_max y (H - y) / H^2 with H = ny - 1 (zero on the wall rows)."""
    y = np.arange(ny, dtype=np.float64)
    h = ny - 1.0
    return 4.0 * u_max * y * (h - y) / h ** 2


def channel_classes(nx, ny, inlet=True, outlet=OUTLET_P, periodic_x=False):
    """2D channel: walls on y=0 and y=ny-1, inlet on x=0, outlet on x=nx-1.

    The four corners belong to the walls.
    """
    cls = np.zeros((1, ny, nx), np.uint8)
    if not periodic_x:
        cls[0, :, 0] = INLET if inlet else WALL
        cls[0, :, nx - 1] = outlet
    cls[0, 0, :] = WALL
    cls[0, ny - 1, :] = WALL
    return cls


def small_channel(nx=16, ny=8, *, tau=0.56, cs_smag=0.1, u_in=0.05, profile="uniform",
                  outlet=OUTLET_P, obj_kind=OBJ_DISSIPATION, seed=7, noise_amp=0.3,
                  window_len=20, sample_every=1, ckpt_every=None, g_max=0.5, q_interp=0.1,
                  periodic_x=False, monitor_kind=MON_DRAG, ckpt_format=CKPT_NATIVE,
                  name=None) -> Case:
    """A small 2D channel with walls, inlet, outlet and a noisy design everywhere.

    Used by the parity and adjoint tests: every boundary kind and a nonzero design
    gradient at every node.
    """
    cls = channel_classes(nx, ny, inlet=not periodic_x, outlet=outlet, periodic_x=periodic_x)
    gamma = np.clip(minmax_noise((1, ny, nx), 1.5, seed) * noise_amp, 0.0, 1.0)
    gamma[cls == WALL] = 1.0
    if profile == "parabolic":
        uin = parabolic_profile(ny, u_in)[None, :]
    else:
        uin = np.full((1, ny), u_in)
        uin[0, 0] = uin[0, ny - 1] = 0.0
    if periodic_x:
        uin[:] = 0.0
    w = _objective_weights(obj_kind, cls, gamma, nx, ny, 1)
    uref = (u_in, 0.0, 0.0)
    return Case(name=name or f"channel{nx}x{ny}", lattice=9, nx=nx, ny=ny, nz=1, tau=tau,
                cs_smag=cs_smag, node_class=cls, gamma=gamma, inlet_u=uin, obj_weights=w,
                obj_kind=obj_kind, obj_uref=uref, q_interp=q_interp, g_max=g_max,
                periodic=(1 if periodic_x else 0, 0, 0), monitor_kind=monitor_kind,
                monitor_u=max(u_in, 1e-3), monitor_l=float(ny) / 4, window_len=window_len,
                sample_every=sample_every, ckpt_every=ckpt_every or window_len,
                ckpt_format=ckpt_format, design_box=(1, nx - 1, 1, ny - 1, 0, 1))


def _objective_weights(kind, cls, gamma, nx, ny, nz):
    """Default weights: volume mean over fluid-ish nodes, or the mid-x plane."""
    w = np.zeros((nz, ny, nx))
    if kind == OBJ_DISSIPATION:
        m = gamma < 0.5
        w[m] = 1.0 / m.sum()
    elif kind == OBJ_VELOCITY_DEV:
        xp = (3 * nx) // 4
        w[:, 1:ny - 1, xp] = 1.0 / (ny - 2) / nz
    elif kind == OBJ_PRESSURE:
        xi, xo = 1, nx - 2
        w[:, 1:ny - 1, xi] = 1.0 / ((ny - 2) * nz)
        w[:, 1:ny - 1, xo] = -1.0 / ((ny - 2) * nz)
    elif kind == OBJ_DRAG:
        w[:] = 1.0
    return w


def small_duct3d(nx=10, ny=6, nz=6, *, tau=0.56, cs_smag=0.1, u_in=0.05,
                 outlet=OUTLET_ZG, obj_kind=OBJ_PRESSURE, seed=11, noise_amp=0.3,
                 window_len=12, sample_every=1, ckpt_every=None, periodic_z=False,
                 monitor_kind=MON_DRAG, name=None) -> Case:
    """A small 3D duct (D3Q19): walls on the y and z faces, inlet x=0, outlet x=nx-1."""
    cls = np.zeros((nz, ny, nx), np.uint8)
    cls[:, :, 0] = INLET
    cls[:, :, nx - 1] = outlet
    cls[:, 0, :] = WALL
    cls[:, ny - 1, :] = WALL
    if not periodic_z:
        cls[0, :, :] = WALL
        cls[nz - 1, :, :] = WALL
    gamma = np.clip(minmax_noise((nz, ny, nx), 1.2, seed) * noise_amp, 0.0, 1.0)
    gamma[cls == WALL] = 1.0
    uin = np.zeros((nz, ny))
    face = cls[:, :, 0] == INLET
    uin[face] = u_in
    w = _objective_weights(obj_kind, cls, gamma, nx, ny, nz)
    if obj_kind == OBJ_PRESSURE:
        w[:] = 0.0
        zi = slice(0, nz) if periodic_z else slice(1, nz - 1)
        nsec = (ny - 2) * (nz if periodic_z else nz - 2)
        w[zi, 1:ny - 1, 1] = 1.0 / nsec
        w[zi, 1:ny - 1, nx - 2] = -1.0 / nsec
    z0, z1 = (0, nz) if periodic_z else (1, nz - 1)
    return Case(name=name or f"duct{nx}x{ny}x{nz}", lattice=19, nx=nx, ny=ny, nz=nz, tau=tau,
                cs_smag=cs_smag, node_class=cls, gamma=gamma, inlet_u=uin, obj_weights=w,
                obj_kind=obj_kind, obj_uref=(u_in, 0.0, 0.0), periodic=(0, 0, 1 if periodic_z else 0),
                monitor_kind=monitor_kind, monitor_u=u_in, monitor_l=float(ny - 2),
                window_len=window_len, sample_every=sample_every,
                ckpt_every=ckpt_every or window_len, design_box=(1, nx - 1, 1, ny - 1, z0, z1))


def stack_cases(cases, name=None) -> Case:
    """A batch of independent 2D problems: the D2Q9 cases (same size and
    parameters; designs, weights, inlet profiles and classes may differ) as
    the z-slices of one lattice.  Boxes become the union over the slices."""
    c0 = cases[0]
    assert c0.lattice == 9 and all(c.lattice == 9 and c.nz == 1 and (c.nx, c.ny) == (c0.nx, c0.ny) for c in cases)
    cat = lambda a: np.concatenate([getattr(c, a) for c in cases], axis=0)
    b = list(c0.design_box)
    b[4], b[5] = 0, len(cases)
    return c0.replace(name=name or f"{c0.name}x{len(cases)}", nz=len(cases), node_class=cat("node_class"),
                      gamma=cat("gamma"), obj_weights=cat("obj_weights"), inlet_u=cat("inlet_u"),
                      design_box=tuple(b), periodic=(c0.periodic[0], c0.periodic[1], 0))


def periodic_box(nx, ny, nz=1, *, lattice=9, tau=0.6, cs_smag=0.0, gamma=None):
    """Fully periodic domain (no boundary nodes); used for invariance tests."""
    cls = np.zeros((nz, ny, nx), np.uint8)
    g = np.zeros((nz, ny, nx)) if gamma is None else np.asarray(gamma, np.float64)
    return Case(name=f"periodic{nx}x{ny}x{nz}", lattice=lattice, nx=nx, ny=ny, nz=nz, tau=tau,
                cs_smag=cs_smag, node_class=cls, gamma=g, inlet_u=np.zeros((nz, ny)),
                obj_weights=np.full((nz, ny, nx), 1.0 / (nx * ny * nz)), obj_kind=OBJ_DISSIPATION,
                periodic=(1, 1, 1 if nz > 1 else 0), monitor_kind=MON_OBJECTIVE,
                design_box=(0, nx, 0, ny, 0, nz))


# ---------------------------------------------------------------------------
# The five workload shapes (seed = 1000 + index).
# ---------------------------------------------------------------------------

def config_channel(seed=1001) -> Case:
    """D2Q9 128x64 channel, parabolic inlet u_max=0.05, zero-gradient outlet,
    disk D=16 at (32,32) plus smooth noise (amplitude 0.05, sigma 3), Re=100 on D,
    Cs=0.1, windows of 200 steps sampled every step, mean viscous dissipation."""
    nx, ny = 128, 64
    cls = channel_classes(nx, ny, outlet=OUTLET_ZG)
    gamma = disk_mask(nx, ny, 32, 32, 16).astype(np.float64)[None]
    gamma = np.clip(gamma + scaled_noise((1, ny, nx), 3.0, 0.05, seed), 0.0, 1.0)
    gamma[cls == WALL] = 1.0
    uin = parabolic_profile(ny, 0.05)[None, :]
    m = gamma < 0.5
    w = np.where(m, 1.0 / m.sum(), 0.0)
    return Case(name="channel128x64", lattice=9, nx=nx, ny=ny, nz=1,
                tau=tau_from_re(0.05, 16, 100), cs_smag=0.1, node_class=cls, gamma=gamma,
                inlet_u=uin, obj_weights=w, obj_kind=OBJ_DISSIPATION, monitor_u=0.05,
                monitor_l=16.0, window_len=200, sample_every=1, conv_tol=1e-3,
                ckpt_every=200, max_windows=10, design_box=(1, nx - 1, 1, ny - 1, 0, 1))


def config_cylinder(re=51.2) -> Case:
    """D2Q9 200x100 flow around a circular cylinder (the cylinder case of Sec. 4):
    radius 8 at the domain centre with phi = 0.5 inside (gamma = 0.5), Re = 51.2
    on the diameter by default (vortex shedding), uniform inlet u = 0.04 (the
    paper gives no inlet speed), Zou-He pressure outlet, walls y = 0 and 99;
    objective = the drag on the body over the design domain, the 32x32 square
    around the cylinder: weights -1 on Eq. 44's F_x, the x-momentum the
    partial bounce-back gives the fluid (negative for flow in +x), so that
    minimising J reduces the drag; windows of 5000 steps sampled every 50
    (Delta W), checkpoints every 100, tolerance 1e-3 on the drag monitor."""
    nx, ny = 200, 100
    cls = channel_classes(nx, ny, outlet=OUTLET_P)
    gamma = np.where(disk_mask(nx, ny, 100, 50, 16), 0.5, 0.0)[None]
    gamma[cls == WALL] = 1.0
    uin = np.full((1, ny), 0.04)
    uin[0, 0] = uin[0, ny - 1] = 0.0
    box = (84, 116, 34, 66)
    w = np.zeros((1, ny, nx))
    w[0, box[2]:box[3], box[0]:box[1]] = -1.0
    return Case(name="cylinder200x100", lattice=9, nx=nx, ny=ny, nz=1,
                tau=tau_from_re(0.04, 16, re), cs_smag=0.1, node_class=cls, gamma=gamma,
                inlet_u=uin, obj_weights=w, obj_kind=OBJ_DRAG, monitor_kind=MON_DRAG,
                monitor_u=0.04, monitor_l=16.0, window_len=5000, sample_every=50,
                conv_tol=1e-3, ckpt_every=100, max_windows=12,
                design_box=(box[0], box[1], box[2], box[3], 0, 1))


def config_wake(seed=1002) -> Case:
    """D2Q9 1024x256 cylinder wake: disk D=32 at (256,128), Re=200, uniform inlet
    u=0.04, Zou-He pressure outlet; design = min-max smooth noise (sigma 6) in
    x in [272,528), y in [64,192); objective = mean squared deviation of u from
    the inflow on the plane x=900; windows of 2000 steps, checkpoints every 100."""
    nx, ny = 1024, 256
    cls = channel_classes(nx, ny, outlet=OUTLET_P)
    gamma = disk_mask(nx, ny, 256, 128, 32).astype(np.float64)[None]
    box = (272, 528, 64, 192)
    gamma[0, box[2]:box[3], box[0]:box[1]] = np.maximum(
        gamma[0, box[2]:box[3], box[0]:box[1]],
        minmax_noise((box[3] - box[2], box[1] - box[0]), 6.0, seed))
    gamma[cls == WALL] = 1.0
    uin = np.full((1, ny), 0.04)
    uin[0, 0] = uin[0, ny - 1] = 0.0
    w = np.zeros((1, ny, nx))
    w[0, 1:ny - 1, 900] = 1.0 / (ny - 2)
    return Case(name="wake1024x256", lattice=9, nx=nx, ny=ny, nz=1,
                tau=tau_from_re(0.04, 32, 200), cs_smag=0.1, node_class=cls, gamma=gamma,
                inlet_u=uin, obj_weights=w, obj_kind=OBJ_VELOCITY_DEV, obj_uref=(0.04, 0.0, 0.0),
                monitor_u=0.04, monitor_l=32.0, window_len=2000, sample_every=1,
                conv_tol=1e-3, ckpt_every=100, max_windows=20,
                design_box=(box[0], box[1], box[2], box[3], 0, 1))


def config_step(seed=1003, ckpt_format=CKPT_FP16) -> Case:
    """D2Q9 2048x512 backward-facing step: solid block x<400, y<128; walls y=0,511;
    uniform inlet u=0.05 above the step; Zou-He pressure outlet; Re=800 on the step
    height, Cs=0.12; noise (sigma 8, amplitude 0.1) over the whole domain;
    windows of 2500 steps, 16-bit checkpoints every 250 steps; objective = mean
    pressure drop between the sections x=8 and x=nx-9."""
    nx, ny, hs = 2048, 512, 128
    cls = channel_classes(nx, ny, outlet=OUTLET_P)
    cls[0, 1:hs + 1, 0] = WALL
    gamma = np.zeros((1, ny, nx))
    gamma[0, :hs, :400] = 1.0
    gamma = np.clip(gamma + scaled_noise((1, ny, nx), 8.0, 0.1, seed), 0.0, 1.0)
    gamma[cls == WALL] = 1.0
    uin = np.zeros((1, ny))
    uin[0, hs + 1:ny - 1] = 0.05
    w = np.zeros((1, ny, nx))
    w[0, hs + 1:ny - 1, 8] = 1.0 / (ny - 2 - hs)
    w[0, 1:ny - 1, nx - 9] = -1.0 / (ny - 2)
    return Case(name="step2048x512", lattice=9, nx=nx, ny=ny, nz=1,
                tau=tau_from_re(0.05, hs, 800), cs_smag=0.12, node_class=cls, gamma=gamma,
                inlet_u=uin, obj_weights=w, obj_kind=OBJ_PRESSURE, monitor_u=0.05,
                monitor_l=float(hs), window_len=2500, sample_every=1, conv_tol=1e-3,
                ckpt_every=250, ckpt_format=ckpt_format, max_windows=40,
                design_box=(0, nx, 1, ny - 1, 0, 1))


def ubend_geometry(nx, ny, nz, lf):
    """Solid mask, node classes and sections of a U-bend duct on the x=0 face.

    Legs of width lf run along x; the upper leg is the inlet, the lower the
    outlet; a half-annulus (inner radius lf/2, outer lf/2+lf) joins them at
    x = xr.  The duct's z-extent is nz - 2*ld with ld = lf/2.
    """
    ld = lf // 2
    lm = lf
    r_in, r_out = lm / 2.0, lm / 2.0 + lf
    xr = nx - int(r_out) - ld
    yc = ny / 2.0
    z, y, x = np.mgrid[0:nz, 0:ny, 0:nx]
    zc0, zc1 = ld, nz - ld
    inz = (z >= zc0) & (z < zc1)
    upper = (y >= yc + r_in) & (y < yc + r_out) & (x < xr)
    lower = (y >= yc - r_out) & (y < yc - r_in) & (x < xr)
    rr = np.sqrt((x + 0.5 - xr) ** 2 + (y + 0.5 - yc) ** 2)
    bend = (x >= xr) & (rr >= r_in) & (rr < r_out)
    fluid = inz & (upper | lower | bend)
    cls = np.zeros((nz, ny, nx), np.uint8)
    face = (x == 0) | (x == nx - 1) | (y == 0) | (y == ny - 1) | (z == 0) | (z == nz - 1)
    cls[face] = WALL
    inl = (x == 0) & inz & upper & (y > yc + r_in) & (y < yc + r_out - 1)
    inl &= (z > zc0) & (z < zc1 - 1)
    outl = (x == 0) & inz & lower & (y > yc - r_out) & (y < yc - r_in - 1)
    outl &= (z > zc0) & (z < zc1 - 1)
    cls[inl] = INLET
    cls[outl] = OUTLET_ZG
    return fluid, cls, xr, ld


def ubend_case(nx, ny, nz, lf, *, re=1000.0, tau=None, cs_smag=0.1, u_in=0.05, window_len=1000,
               ckpt_every=200, ckpt_format=CKPT_BF16, seed=1004, name=None) -> Case:
    """A D3Q19 U-bend duct (ubend_geometry) with a velocity inlet on its upper
    leg and a zero-gradient outlet on its lower leg, both on the x = 0 face.
    Design = smooth noise (sigma 4) in the bend region x >= xr; objective =
    mean pressure drop between the inlet and outlet legs at x = lf; tau from
    Re on the leg width unless given."""
    fluid, cls, xr, ld = ubend_geometry(nx, ny, nz, lf)
    gamma = np.where(fluid, 0.0, 1.0)
    region = np.zeros_like(fluid)
    region[:, :, xr:] = True
    noise = minmax_noise((nz, ny, nx), 4.0, seed)
    gamma = np.where(fluid & region, 0.6 * noise * (noise > 0.5), gamma)
    gamma[cls == WALL] = 1.0
    gamma[cls == INLET] = 0.0
    gamma[cls == OUTLET_ZG] = 0.0
    uin = np.where(cls[:, :, 0] == INLET, u_in, 0.0)
    w = np.zeros((nz, ny, nx))
    lp = lf
    sec_in = fluid[:, :, lp] & (np.mgrid[0:nz, 0:ny][1] > ny / 2)
    sec_out = fluid[:, :, lp] & (np.mgrid[0:nz, 0:ny][1] < ny / 2)
    w[:, :, lp][sec_in] = 1.0 / sec_in.sum()
    w[:, :, lp][sec_out] = -1.0 / sec_out.sum()
    return Case(name=name or f"ubend{nx}x{ny}x{nz}", lattice=19, nx=nx, ny=ny, nz=nz,
                tau=tau if tau is not None else tau_from_re(u_in, lf, re), cs_smag=cs_smag, node_class=cls,
                gamma=gamma, inlet_u=uin, obj_weights=w, obj_kind=OBJ_PRESSURE, monitor_u=u_in,
                monitor_l=float(lf), window_len=window_len, sample_every=1, conv_tol=1e-3,
                ckpt_every=ckpt_every, ckpt_format=ckpt_format, max_windows=40,
                design_box=(xr, nx - 1, 1, ny - 1, ld, nz - ld))


def config_ubend(seed=1004, big=False) -> Case:
    """D3Q19 U-bend duct.  Small: 256x128x64, lf=32, Re=1000, Cs=0.1, windows of
    1000, BF16 checkpoints every 200.  Big: 384x192x192, lf=48, Re=3000, Cs=0.15,
    windows of 2000, BF16 checkpoints every 50.  Design = smooth noise (sigma 4)
    in the bend region; objective = mean pressure drop between the inlet and
    outlet legs."""
    if big:
        return ubend_case(384, 192, 192, 48, re=3000.0, cs_smag=0.15, window_len=2000, ckpt_every=50, seed=seed)
    return ubend_case(256, 128, 64, 32, re=1000.0, cs_smag=0.1, window_len=1000, ckpt_every=200, seed=seed)


WORKLOADS = {
    "channel128x64": config_channel,
    "cylinder200x100": config_cylinder,
    "wake1024x256": config_wake,
    "step2048x512": config_step,
    "ubend256x128x64": lambda: config_ubend(big=False),
    "ubend384x192x192": lambda: config_ubend(big=True),
}
