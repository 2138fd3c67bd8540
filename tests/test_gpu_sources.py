"""Interface source terms on the GPU against the oracle (componentwise, fp64 bar 1e-12 of the
absolute integrand)."""
import numpy as np
import pytest

import synthetic as syn
from oracle import interface as oi
from problems import componentwise_ok, oseen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

EV = syn.EVAPORATION
TI = syn.TI64


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2501_18781_gb300 import Context, build_library
    build_library()
    return Context(0)


def _evaluate(P, T, model, heaviside, eps, op):
    p = dict(rho_l=TI["rho_l"], rho_g=TI["rho_g"], rhocp_l=TI["rho_l"] * TI["cp_l"], rhocp_g=TI["rho_g"] * TI["cp_g"],
             heaviside=heaviside, eps=eps, model=model, recoil=True, **EV)
    ref = oi.interface_sources(P["dmu"], P["dmp"], P["phi"], T, p)
    bound = oi.interface_sources(P["dmu"], P["dmp"], P["phi"], T, p, absolute=True)
    got = op.interface_sources(torch.tensor(T, device="cuda"), EV["p_amb"], EV["h_v"], EV["molar_mass"],
                               EV["t_boil"], p["rhocp_l"], p["rhocp_g"], mass_flux=model, sticking=EV["sticking"],
                               tanasawa_coef=EV["tanasawa"])
    for key, r, b in zip(("u", "p", "T"), ref, bound):
        ok, worst = componentwise_ok(got[key].cpu().numpy(), r, b, 1e-12)
        assert ok, (key, model, heaviside, worst)
        assert np.abs(r).max() > 0
    return got


@pytest.mark.parametrize("model", ["knight", "tanasawa"])
def test_interface_sources_match_oracle(ctx, model):
    P = oseen(6, ctx)
    T = syn.interface_temperature(*P["dmu"].dof_coords().T)
    wl = syn.scaled(syn.OSEEN_INTERFACE, 6)
    got = _evaluate(P, T, model, "tanh", wl.eps, P["op"])
    assert np.all(got["u"].cpu().numpy()[np.tile(P["dmu"].dirichlet, 3)] == 0.0)


def test_interface_sources_sine_heaviside(ctx):
    from paper_2501_18781_gb300 import Operator
    P = oseen(5, ctx)
    wl = syn.scaled(syn.OSEEN_INTERFACE, 5)
    p = wl.params
    op = Operator(ctx, "oseen", list(P["maps"]), sigma=P["sigma"], rho_l=p["rho_l"], rho_g=p["rho_g"],
                  mu_l=p["mu_l"], mu_g=p["mu_g"], eps=wl.eps, heaviside=1)
    op.set_field("phi", torch.tensor(P["phi"], device="cuda"))
    op.set_field("beta", torch.tensor(P["beta"].ravel(), device="cuda"))
    T = syn.interface_temperature(*P["dmu"].dof_coords().T)
    _evaluate(P, T, "knight", "sine", wl.eps, op)


def test_interface_sources_reject_other_operators(ctx):
    from paper_2501_18781_gb300._lib import MFError
    from problems import helmholtz
    P = helmholtz(3, ctx)
    with pytest.raises(MFError):
        P["op"].interface_sources(torch.zeros(P["n"], dtype=torch.float64, device="cuda"), 1e5, 1e6, 0.05, 3000.0,
                                  1.0, 1.0)
