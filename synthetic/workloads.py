"""Named synthetic workloads shaped like the paper's melt-pool problems.

Material constants are the Ti-6Al-4V table of Section 4.3 (Table tab:param_ti64); the
domain [-300, 300] um^3 and the laser absorptivity 0.35 follow Section 4.3.  The sizes
and the coefficient recipes are the five benchmark workloads of this library.
"""
from dataclasses import dataclass, field, replace
from typing import Tuple

TI64 = dict(
    rho_l=4087.0, rho_g=4.087,          # kg/m^3
    mu_l=3.5e-3, mu_g=3.5e-5,           # kg/(m s)
    cp_l=1130.0, cp_g=11.3,             # J/(kg K)
    k_l=28.63, k_g=0.02863,             # W/(m K)
    t_boil=3133.0,                      # K
    molar_mass=4.78e-2,                 # kg/mol
    h_v=8.84e6,                         # J/kg, latent heat of evaporation
    sticking=1.0,                       # c_s
)

# Evaporation inputs of the interface source terms: the Ti-6Al-4V values above, atmospheric
# ambient pressure, and a Tanasawa coefficient for the linear mass-flux law.
EVAPORATION = dict(p_amb=101325.0, h_v=TI64["h_v"], molar_mass=TI64["molar_mass"], t_boil=TI64["t_boil"],
                   sticking=TI64["sticking"], tanasawa=1e-3)


@dataclass(frozen=True)
class Workload:
    name: str
    kind: str                      # helmholtz | oseen | heat | heat_adjoint | reinit
    n: int                         # cells per axis (uniform) or base cells per axis (octree)
    lo: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    hi: Tuple[float, float, float] = (1.0, 1.0, 1.0)
    degree: int = 2
    levels: int = 0                # octree refinement levels
    nrhs: int = 1
    seed: int = 1
    params: dict = field(default_factory=dict)

    @property
    def h(self):
        return (self.hi[0] - self.lo[0]) / (self.n << self.levels)

    @property
    def eps(self):
        """Interface thickness parameter eps = 2 h_finest (Section 3.1 choice eps = 2h)."""
        return 2.0 * self.h


HELMHOLTZ_SPHERE = Workload(
    "helmholtz_sphere_q2_16", "helmholtz", 16,
    params=dict(mass=1.0, a_gas=1.0, a_liquid=1000.0, sphere_radius=0.3, tol=1e-10))

OSEEN_INTERFACE = Workload(
    "oseen_q2q1_interface_64", "oseen", 64,
    params=dict(rho_l=TI64["rho_l"], rho_g=TI64["rho_g"], mu_l=TI64["mu_l"], mu_g=TI64["mu_g"],
                dt_cfl=0.5, restart=50, tol=1e-10, maxit=5000))

_LASER = dict(power=200.0, radius=50e-6, x0=0.0, y0=0.0, absorptivity=0.35)

HEAT_LASER = Workload(
    "heat_laser_q2_128", "heat", 128, lo=(-3e-4, -3e-4, -3e-4), hi=(3e-4, 3e-4, 3e-4),
    params=dict(rhocp=TI64["rho_l"] * TI64["cp_l"], k0=TI64["k_l"], t_boil=TI64["t_boil"],
                dt=1e-5, t_ref=500.0, laser=_LASER, cheby_degree=4, tol=1e-10))

HEAT_ADJOINT = Workload(
    "heat_adjoint_q2_64", "heat_adjoint", 64, lo=(-3e-4, -3e-4, -3e-4), hi=(3e-4, 3e-4, 3e-4),
    params=dict(rhocp=TI64["rho_l"] * TI64["cp_l"], k0=TI64["k_l"], t_boil=TI64["t_boil"],
                dt=1e-5, t_ref=500.0, laser=_LASER, box_half=100e-6, box_depth=100e-6,
                fd_step=1e-6, tol=1e-12))

REINIT_OCTREE = Workload(
    "reinit_octree_q2_32_l3", "reinit", 32, levels=3, nrhs=8,
    params=dict(sphere_radius=0.3, amplitude=0.05, lmax=6, tol=1e-10))


# One step of the melt-pool algorithm on the 600 um box of Section 4.3 at the paper's time step of
# 0.01 us: there the Darcy damping C = 1e12 is 2.45 rho_l / dt and the gas-side transport velocity
# mdot / rho_g (tens of m/s near the boiling point) moves the interface 0.06 cells per step.
MELTPOOL_STEP = Workload(
    "meltpool_step_q2q1_64", "meltpool_step", 64, lo=(-3e-4, -3e-4, -3e-4), hi=(3e-4, 3e-4, 3e-4),
    params=dict(dt=1e-8, u_max=1.0, reinit_steps=2, dtau_cells=0.5,
                laser=dict(power=200.0, radius=50e-6, absorptivity=0.35, focus=(0.0, 0.0, 0.0),
                           direction=(0.0, 0.0, -1.0)),
                surface_tension=dict(alpha0=1.493, alpha1=5.5e-4, t_alpha=1928.0, alpha_res=0.01),
                gravity=(0.0, 0.0, -9.81),
                solid=dict(rho_s=TI64["rho_l"], mu_s=TI64["mu_l"], t_solidus=1933.0, t_liquidus=2200.0),
                darcy=dict(C=1e12, b=1.0, t_solidus=1933.0, t_liquidus=2200.0),
                trace_correction=True, tol=1e-10, flow_tol=1e-10,
                # solver settings measured best on the 64^3 step (reinit by fp32-inner defect
                # correction; flow preconditioner: 5 velocity GMRES steps, Schur CG to 0.1 or 30 steps)
                reinit_mixed=1, flow_velocity_steps=5, flow_schur_maxit=30, flow_schur_tol=0.1))


def scaled(wl, n, levels=None, nrhs=None):
    """The same workload recipe on a smaller (or larger) mesh."""
    kw = dict(n=n, name=f"{wl.name}@n{n}")
    if levels is not None:
        kw["levels"] = levels
    if nrhs is not None:
        kw["nrhs"] = nrhs
    return replace(wl, **kw)
