"""Seeded synthetic inputs for the RFA bioheat path.

This module produces only *inputs*: voxel label volumes, per-label tissue
tables in SI units, needle descriptions and grid/time parameters.  It holds
none of the method's arithmetic (no coefficients, no source field, no time
stepping), so both the CUDA path and the FP64 oracle can consume its output
without sharing any computation.

The paper simulated a segmented patient CT (Sec. "Implementation": 256^2 x 234
voxels) and Linte's in-vitro set-up (Sec. "Evaluation Methods"); neither is
available, so seeded phantoms with the same kind of structure stand in:
a liver background, spherical tumours and cylindrical vessels held at blood
temperature (Sec. "Specialized Methods": vessels keep 37 C).

Generator recipe (all draws from ``numpy.random.default_rng(seed)`` in the
order listed in ``tumor_vessel_phantom``):
  1. n_tumors ~ U{1..3}; each radius ~ U(5, 15) mm, centre uniform in the
     central 50 % box of the grid.
  2. needle tip uniform in a ball of 0.5 r around tumour 0's centre
     (single-needle configurations) or grid centre +- 5 mm (batched members).
  3. n_vessels ~ U{2..4} (or a fixed count); each radius ~ U(1, 3) mm, a line
     through a uniform point of the box with an isotropic direction; a line
     whose distance to the tip is below r_v + 3 mm + needle reach is redrawn.
  4. label precedence: vessel > tumour > liver.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

# Label ids used by every generator in this module.
LIVER, TUMOR, VESSEL = 0, 1, 2

# Needle kinds (same numbering as the C header).
STRAIGHT, UMBRELLA, FIXED_TIP = 0, 1, 2

# Face boundary modes (same numbering as the C header).
DIRICHLET, INSULATED = 0, 1


@dataclasses.dataclass
class Tissue:
    """Per-label physical parameters in SI units (Eq. 2675-eq1_Kath symbols)."""
    k: float = 0.52          # thermal conductivity K [W/m/K]
    rho: float = 1060.0      # tissue density [kg/m^3]
    c: float = 3600.0        # tissue heat capacity c_p [J/kg/K]
    w_b: float = 6.4e-3      # perfusion rate [1/s]
    rho_b: float = 1000.0    # blood density [kg/m^3]
    c_b: float = 4180.0      # blood heat capacity [J/kg/K]
    Q_m: float = 0.0         # metabolic heat [W/m^3]
    fixed: int = 0           # 1: voxel held at T_fixed_C (vessel / hot tip)
    T_fixed_C: float = 37.0
    sigma: float = 0.33      # electrical conductivity [S/m] (potential-solve source only)

    def as_tuple(self):
        return (self.k, self.rho, self.c, self.w_b, self.rho_b, self.c_b,
                self.Q_m, int(self.fixed), self.T_fixed_C)


def liver() -> Tissue:
    return Tissue()


def tumor() -> Tissue:
    return Tissue(k=0.55, w_b=3e-3, sigma=0.45)


def vessel() -> Tissue:
    return Tissue(fixed=1, T_fixed_C=37.0, sigma=0.7)


def paper_liver() -> Tissue:
    """The liver values printed with Eq. 2675-eq1_Kath (Q_m = 10714 W/m^3,
    rho = 1079, c_p = 3540, K = 0.52, w_b c_b = 16.687 * 3617 with rho_b = 1)."""
    return Tissue(k=0.52, rho=1079.0, c=3540.0, w_b=16.687, rho_b=1.0,
                  c_b=3617.0, Q_m=10714.0)


def default_table() -> List[Tissue]:
    return [liver(), tumor(), vessel()]


@dataclasses.dataclass
class Needle:
    """Needle description; positions in metres, grid voxel (i,j,k) sits at (i*h, j*h, k*h)."""
    kind: int = STRAIGHT
    tip: Sequence[float] = (0.0, 0.0, 0.0)
    axis: Sequence[float] = (0.0, 0.0, 1.0)
    active_len: float = 15e-3       # straight: active length behind the tip
    tine_len: float = 10e-3         # umbrella: tine length
    tine_polar_deg: float = 60.0    # umbrella: angle of the tines off the axis
    n_tines: int = 4                # umbrella: tines on the ring
    tine_axial: int = 0             # umbrella: 1 adds a tine along the axis
    power: float = 15.0             # RF power [W]
    r_clamp: float = 1e-3           # 1/r^4 clamp radius r0 [m]
    T_tip_C: float = 90.0           # FIXED_TIP mode temperature

    def reach(self) -> float:
        if self.kind == STRAIGHT:
            return self.active_len
        if self.kind == UMBRELLA:
            return self.tine_len
        return 3e-3


@dataclasses.dataclass
class Damage:
    """Arrhenius constants (Eq. eq-tissState) and the necrosis threshold."""
    enable: int = 1
    A: float = 7.39e39
    Ea: float = 2.577e5
    R: float = 8.31
    T_thr_C: float = 60.0


@dataclasses.dataclass
class Case:
    """One simulation problem: grid, tissue labels, table, needle, time stepping."""
    name: str
    nx: int
    ny: int
    nz: int
    h: float
    dt: float
    nsteps: int
    labels: np.ndarray              # uint8 [nz][ny][nx], x fastest
    table: List[Tissue]
    needle: Needle
    damage: Damage
    T_a_C: float = 37.0
    face_bc: int = DIRICHLET
    conduction: str = "centre"      # "centre" (K at the voxel) or "harmonic" (conservative)
    source: str = "needle"          # "needle" (max(d, r0)^-4) or "potential" (sigma |grad V|^2)
    perfusion: str = "constant"     # "constant" or "tissue_state" (w_b weighted by 1/max(1, Omega))

    @property
    def nvox(self) -> int:
        return self.nx * self.ny * self.nz


def centre(n: int, h: float) -> float:
    """Physical coordinate of the grid centre when voxel i sits at i*h."""
    return 0.5 * (n - 1) * h


def straight_through_centre(n: int, h: float, active_len: float, power: float) -> Needle:
    """Straight needle along +z through the grid centre; the active part is
    centred on the grid centre and the tip is its distal (+z) end."""
    c = centre(n, h)
    return Needle(kind=STRAIGHT, tip=(c, c, c + 0.5 * active_len), axis=(0.0, 0.0, 1.0),
                  active_len=active_len, power=power)


def homogeneous_case(n: int = 64, h: float = 1e-3, dt: float = 0.05, nsteps: int = 2000,
                     active_len: float = 15e-3, power: float = 15.0,
                     damage: Optional[Damage] = None, name: str = "homogeneous") -> Case:
    """Homogeneous liver, Dirichlet 37 C faces, straight needle through the centre
    (64^3, h = 1 mm, 15 mm active, 15 W, dt = 0.05 s, 2000 steps by default)."""
    labels = np.zeros((n, n, n), dtype=np.uint8)
    dmg = damage if damage is not None else Damage(enable=0)
    return Case(name=name, nx=n, ny=n, nz=n, h=h, dt=dt, nsteps=nsteps, labels=labels,
                table=default_table(), needle=straight_through_centre(n, h, active_len, power),
                damage=dmg)


def _unit(v):
    v = np.asarray(v, dtype=np.float64)
    return v / np.linalg.norm(v)


def _point_line_distance(p, a, d):
    """Distance from point p to the infinite line a + t d (|d| = 1)."""
    w = np.asarray(p, dtype=np.float64) - a
    return float(np.linalg.norm(w - np.dot(w, d) * d))


def paint_labels(nx, ny, nz, h, tumors, vessels, z_chunk: int = 64) -> np.ndarray:
    """Rasterise spheres (tumours) and infinite cylinders (vessels) at voxel
    centres, vessel > tumour > liver.  Spheres are painted inside their bounding
    boxes; cylinders per z-chunk; coordinates in float32."""
    labels = np.zeros((nz, ny, nx), dtype=np.uint8)
    f = np.float32
    for (cx, cy, cz, r) in tumors:
        lo = [max(0, int(np.floor((c - r) / h))) for c in (cz, cy, cx)]
        hi = [min(n, int(np.ceil((c + r) / h)) + 1) for c, n in ((cz, nz), (cy, ny), (cx, nx))]
        if any(a >= b for a, b in zip(lo, hi)):
            continue
        zs = (np.arange(lo[0], hi[0], dtype=f) * f(h) - f(cz))[:, None, None]
        ys = (np.arange(lo[1], hi[1], dtype=f) * f(h) - f(cy))[None, :, None]
        xs = (np.arange(lo[2], hi[2], dtype=f) * f(h) - f(cx))[None, None, :]
        inside = zs * zs + ys * ys + xs * xs <= f(r * r)
        labels[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]][inside] = TUMOR
    xs = np.arange(nx, dtype=f) * f(h)
    ys = np.arange(ny, dtype=f) * f(h)
    for (a, d, r) in vessels:
        a = np.asarray(a, dtype=np.float64)
        d = np.asarray(d, dtype=np.float64)
        wx = (xs - f(a[0]))[None, None, :]
        wy = (ys - f(a[1]))[None, :, None]
        for z0 in range(0, nz, z_chunk):
            z1 = min(nz, z0 + z_chunk)
            wz = (np.arange(z0, z1, dtype=f) * f(h) - f(a[2]))[:, None, None]
            t = wx * f(d[0]) + wy * f(d[1]) + wz * f(d[2])
            # squared distance to the axis = |w|^2 - t^2
            dist2 = wx * wx + wy * wy + wz * wz - t * t
            labels[z0:z1][dist2 <= f(r * r)] = VESSEL
    return labels


def tumor_vessel_phantom(nx: int, ny: int, nz: int, h: float, rng: np.random.Generator,
                         needle_fn, n_vessels: Optional[int] = None,
                         tip_mode: str = "tumor"):
    """Draw tumours, the needle (via ``needle_fn(tip)``) and vessels in the
    documented order; return (labels, needle, tumors, vessels)."""
    L = np.array([nx, ny, nz], dtype=np.float64) * h
    lo, hi = 0.25 * L, 0.75 * L
    nt = int(rng.integers(1, 4))
    tumors = []
    for _ in range(nt):
        r = float(rng.uniform(5e-3, 15e-3))
        c = rng.uniform(lo, hi)
        tumors.append((float(c[0]), float(c[1]), float(c[2]), r))
    if tip_mode == "tumor":
        cx, cy, cz, r = tumors[0]
        while True:
            u = rng.uniform(-1.0, 1.0, size=3)
            if np.dot(u, u) <= 1.0:
                break
        tip = np.array([cx, cy, cz]) + 0.5 * r * u
    else:
        gc = np.array([centre(nx, h), centre(ny, h), centre(nz, h)])
        tip = gc + rng.uniform(-5e-3, 5e-3, size=3)
    needle = needle_fn(tuple(float(t) for t in tip))
    nv = int(rng.integers(2, 5)) if n_vessels is None else int(n_vessels)
    vessels = []
    for _ in range(nv):
        r = float(rng.uniform(1e-3, 3e-3))
        for _try in range(1000):
            a = rng.uniform(np.zeros(3), L)
            d = _unit(rng.normal(size=3))
            if _point_line_distance(tip, a, d) > r + 3e-3 + needle.reach():
                vessels.append((a, d, r))
                break
    labels = paint_labels(nx, ny, nz, h, tumors, vessels)
    return labels, needle, tumors, vessels


def single_needle_case(seed: int = 0, n: int = 256, h: float = 0.5e-3, dt: float = 0.05,
                       nsteps: int = 12000, power: float = 30.0, kind: int = UMBRELLA,
                       n_tines: int = 4, tine_axial: int = 0, tine_len: float = 10e-3,
                       active_len: float = 15e-3, n_vessels: Optional[int] = None,
                       damage: Optional[Damage] = None, name: str = "single") -> Case:
    """Tumour + vessel phantom with one needle whose tip lies in tumour 0.
    Defaults: 256^3, h = 0.5 mm, 4-tine umbrella (10 mm tines), 30 W,
    dt = 0.05 s, 12000 steps, Arrhenius damage on."""
    rng = np.random.default_rng(seed)

    def needle_fn(tip):
        return Needle(kind=kind, tip=tip, axis=(0.0, 0.0, 1.0), active_len=active_len,
                      tine_len=tine_len, n_tines=n_tines, tine_axial=tine_axial, power=power)

    labels, needle, _, _ = tumor_vessel_phantom(n, n, n, h, rng, needle_fn, n_vessels=n_vessels)
    return Case(name=name, nx=n, ny=n, nz=n, h=h, dt=dt, nsteps=nsteps, labels=labels,
                table=default_table(), needle=needle,
                damage=damage if damage is not None else Damage())


def umbrella_case_256(seed: int = 0, nsteps: int = 12000) -> Case:
    """256^3, h = 0.5 mm, 1-3 tumours, 2-4 vessels, 4-tine umbrella at 30 W,
    dt = 0.05 s, 12000 steps, BF16 parameter fields, FP64 Arrhenius damage."""
    return single_needle_case(seed=seed, nsteps=nsteps, name="umbrella256")


def adjoint_case_128(seed: int = 0, nsteps: int = 2000) -> Case:
    """128^3, h = 0.75 mm, tumour + vessel phantom, straight 15 mm needle at 20 W,
    dt = 0.05 s, 2000 steps (damage off; the loss uses the final temperature)."""
    return single_needle_case(seed=seed, n=128, h=0.75e-3, nsteps=nsteps, power=20.0,
                              kind=STRAIGHT, damage=Damage(enable=0), name="adjoint128")


def adjoint_case_256(seed: int = 0, nsteps: int = 2000) -> Case:
    """The adjoint workload at the single-needle size: 256^3, h = 0.5 mm, tumour +
    vessel phantom, straight 15 mm needle at 20 W, dt = 0.05 s, 2000 steps
    (damage off); its fields (~0.8 GB) do not fit in L2."""
    return single_needle_case(seed=seed, n=256, h=0.5e-3, nsteps=nsteps, power=20.0,
                              kind=STRAIGHT, damage=Damage(enable=0), name="adjoint256")


def large_case_512(seed: int = 0, nsteps: int = 5000) -> Case:
    """512^3, h = 0.25 mm, 8 vessels, 9-tine umbrella (8 ring + 1 axial) at 40 W,
    dt = 0.02 s, 5000 steps, Arrhenius damage on."""
    return single_needle_case(seed=seed, n=512, h=0.25e-3, dt=0.02, nsteps=nsteps, power=40.0,
                              kind=UMBRELLA, n_tines=8, tine_axial=1, n_vessels=8,
                              name="large512")


def batch_members(seed: int = 0, n_members: int = 64, nsteps: int = 4000,
                  sizes=(96, 128, 160, 192)) -> List[Case]:
    """Uneven batch: grid edge from ``sizes``, h ~ U(0.5, 1) mm, straight
    (10-30 mm active) or 4-/9-tine umbrella (10 mm tines), tip at grid centre
    +- 5 mm, P ~ U(10, 40) W, tumour + vessel phantom, dt = 0.05 s."""
    rng = np.random.default_rng(seed)
    out = []
    for m in range(n_members):
        n = int(rng.choice(sizes))
        h = float(rng.uniform(0.5e-3, 1e-3))
        geo = int(rng.integers(0, 3))
        P = float(rng.uniform(10.0, 40.0))
        act = float(rng.uniform(10e-3, 30e-3))

        def needle_fn(tip, geo=geo, P=P, act=act):
            if geo == 0:
                return Needle(kind=STRAIGHT, tip=tip, active_len=act, power=P)
            if geo == 1:
                return Needle(kind=UMBRELLA, tip=tip, n_tines=4, tine_len=10e-3, power=P)
            return Needle(kind=UMBRELLA, tip=tip, n_tines=8, tine_axial=1, tine_len=10e-3,
                          power=P)

        labels, needle, _, _ = tumor_vessel_phantom(n, n, n, h, rng, needle_fn,
                                                    tip_mode="centre")
        out.append(Case(name=f"member{m}", nx=n, ny=n, nz=n, h=h, dt=0.05, nsteps=nsteps,
                        labels=labels, table=default_table(), needle=needle,
                        damage=Damage(enable=0)))
    return out


def random_small_case(seed: int, nx: int, ny: int, nz: int, h: float = 1e-3, dt: float = 0.05,
                      nsteps: int = 50, kind: int = STRAIGHT, face_bc: int = DIRICHLET,
                      power: float = 15.0, damage: Optional[Damage] = None) -> Case:
    """Small ragged-size phantom for parity tests: random tumour/vessel blobs,
    a needle near the centre."""
    rng = np.random.default_rng(seed)

    def needle_fn(tip):
        if kind == UMBRELLA:
            return Needle(kind=UMBRELLA, tip=tip, n_tines=8, tine_axial=1,
                          tine_len=min(nx, ny, nz) * h * 0.25, power=power)
        return Needle(kind=STRAIGHT, tip=tip, active_len=min(nx, ny, nz) * h * 0.3, power=power)

    L = np.array([nx, ny, nz], dtype=np.float64) * h
    tumors = [(float(x), float(y), float(z), float(rng.uniform(0.1, 0.3) * L.min()))
              for (x, y, z) in rng.uniform(0.3 * L, 0.7 * L, size=(2, 3))]
    tip = 0.5 * (L - h) + rng.uniform(-1.0, 1.0, size=3) * h
    needle = needle_fn(tuple(float(t) for t in tip))
    vessels = []
    for _ in range(2):
        r = float(rng.uniform(0.5, 1.5) * h)
        for _try in range(200):
            a = rng.uniform(np.zeros(3), L)
            d = _unit(rng.normal(size=3))
            if _point_line_distance(tip, a, d) > r + 2 * h + needle.reach():
                vessels.append((a, d, r))
                break
    labels = paint_labels(nx, ny, nz, h, tumors, vessels)
    return Case(name=f"small{nx}x{ny}x{nz}", nx=nx, ny=ny, nz=nz, h=h, dt=dt, nsteps=nsteps,
                labels=labels, table=default_table(), needle=needle,
                damage=damage if damage is not None else Damage(), face_bc=face_bc)


def paper_tip_case(T_tip_C: float = 90.0, n: int = 64, nsteps: int = 1200) -> Case:
    """The paper's evaluation set-up (Sec. "Evaluation Methods"): 0.5 mm voxels,
    a needle tip modelled as a voxel hemisphere five voxels across in x and y
    and three voxels deep in z, held at T_tip (90 or 60 C), time step 0.1 s,
    liver with the paper's printed constants (Q_m = 10714 W/m^3); no RF source.
    Label 1 is the tip.  Probe voxels: see paper_tip_probes()."""
    h = 0.5e-3
    labels = np.zeros((n, n, n), dtype=np.uint8)
    c = n // 2
    for dz in range(3):
        for dy in range(-2, 3):
            for dx in range(-2, 3):
                if (dx / 2.5) ** 2 + (dy / 2.5) ** 2 + (dz / 3.0) ** 2 <= 1.0:
                    labels[c + dz, c + dy, c + dx] = 1
    tip = Tissue(fixed=1, T_fixed_C=T_tip_C)
    return Case(name=f"papertip{int(T_tip_C)}", nx=n, ny=n, nz=n, h=h, dt=0.1, nsteps=nsteps,
                labels=labels, table=[paper_liver(), tip], needle=Needle(kind=STRAIGHT, power=0.0),
                damage=Damage(enable=0, T_thr_C=42.5))


def paper_tip_needle_case(T_tip_C: float = 90.0, n: int = 64, nsteps: int = 1200) -> Case:
    """The same set-up as paper_tip_case, described as the library's FIXED_TIP
    needle instead of a painted label: every voxel is liver (paper constants)
    and the needle's tip sits on the voxel the hemisphere's flat face is
    centred on, axis +z (the dome toward +z)."""
    c = n // 2
    h = 0.5e-3
    base = paper_tip_case(T_tip_C, n, nsteps)
    needle = Needle(kind=FIXED_TIP, tip=(c * h, c * h, c * h), axis=(0.0, 0.0, 1.0), power=0.0,
                    T_tip_C=T_tip_C)
    return Case(name=f"papertipneedle{int(T_tip_C)}", nx=n, ny=n, nz=n, h=h, dt=base.dt, nsteps=nsteps,
                labels=np.zeros((n, n, n), dtype=np.uint8), table=[paper_liver()], needle=needle,
                damage=base.damage)


def paper_tip_probes(n: int = 64):
    """Voxel indices (z, y, x) 2.5 mm and 5 mm beyond the tip's outer x face."""
    c = n // 2
    return {"2.5mm": (c, c, c + 2 + 5), "5mm": (c, c, c + 2 + 10)}



def breathing_field(case: Case, t_s: float, seed: int = 0, period_s: float = 4.0) -> np.ndarray:
    """Synthetic inverse motion vector field u_inv(x, t) of one breathing instant
    (metres, float32 [3][nz][ny][nx]; the paper's fields come from 4D CT, which
    is not available).  Craniocaudal motion along z, strongest above a seeded
    diaphragm level z_d, with a small lateral component:
        s(t)  = sin^2(pi t / period)               (0 at exhale, 1 at inhale)
        w(z)  = (1 + tanh((z - z_d) / L)) / 2,      L = 20 mm
        u_z   = -A s(t) w(z),   u_x = 0.15 A s(t) w(z) sin(pi y / Y),   u_y = 0
    with A ~ U(5, 10) mm.  |du/dx| <= A / (2 L) <= 0.25, so x -> x + u_inv is a
    diffeomorphism."""
    rng = np.random.default_rng(seed)
    A = rng.uniform(5e-3, 10e-3)
    zd = case.h * case.nz * rng.uniform(0.4, 0.6)
    L = 20e-3
    s = math.sin(math.pi * t_s / period_s) ** 2
    z = (np.arange(case.nz) * case.h)[:, None, None]
    y = (np.arange(case.ny) * case.h)[None, :, None]
    Y = max(case.h * (case.ny - 1), case.h)
    w = 0.5 * (1.0 + np.tanh((z - zd) / L))
    u = np.zeros((3, case.nz, case.ny, case.nx), np.float32)
    u[2] = np.broadcast_to(-A * s * w, (case.nz, case.ny, case.nx))
    u[0] = np.broadcast_to(0.15 * A * s * w * np.sin(math.pi * y / Y), (case.nz, case.ny, case.nx))
    return u
