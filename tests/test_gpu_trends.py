"""The trends the paper reports for the steady power-law cavity (Sec. 4.2, 4.3; Tables 3 and 4),
checked on small steady cavities solved by the library: at fixed Ra the heat transfer and the
total entropy generation fall as the power-law index n rises (shear thinning strengthens the
convection), and at fixed n they rise with Ra while the Bejan number falls. Small grids change
the values, not these orderings.

The Bejan number rises with n at Ra = 1e3, as in Table 4. At Ra = 1e4 Table 4 has it rising
steeply with n (0.371, 0.672, 0.849). Here it does not: 0.786, 0.699, 0.701 at 15^3. With the
entropy terms as defined in Sec. 4.3, the heat-transfer integral equals the mean Nusselt
number at steady state, and Nu falls with n. So this ordering is not asserted at Ra = 1e4."""

import pytest

from golden_values import table

pytestmark = pytest.mark.gpu

RAS = (1e2, 1e3, 1e4, 1e5)
TABLE3 = {(Ra, row[0]): row[1 + q] for row in table("table3_total_entropy.txt")
          for q, Ra in enumerate(RAS)}
TABLE4 = {(Ra, row[0]): row[1 + q] for row in table("table4_bejan.txt") for q, Ra in enumerate(RAS)}

H = pytest.importorskip("paper_2411_06563_gb300.hosc")
from paper_2411_06563_gb300 import serve as S  # noqa: E402

N = 15


@pytest.fixture(scope="module")
def steady():
    out = {}
    for Ra in (1e3, 1e4):
        for n in (0.75, 1.0, 1.25):
            p = S.request_params(N, Ra, n, tol_steady=1e-5, tol_div=1e-5)
            with H.Cavity(p) as cav:
                info = cav.solve_steady(200000)
                d = cav.diagnostics()
            assert info["call_status"] == 0, (Ra, n, info)
            out[(Ra, n)] = d
            print("Ra=%g n=%.2f steps=%d Nu_mean=%.4f Nu_max=%.4f E_total=%.4f Be=%.5f" % (
                Ra, n, info["steps"], d["Nu_hot_mean"], d["Nu_hot_max"], d["E_total"], d["Be"]))
    return out


def test_heat_transfer_and_entropy_fall_with_n(steady):
    for Ra in (1e3, 1e4):
        nu = [steady[(Ra, n)]["Nu_hot_mean"] for n in (0.75, 1.0, 1.25)]
        et = [steady[(Ra, n)]["E_total"] for n in (0.75, 1.0, 1.25)]
        be = [steady[(Ra, n)]["Be"] for n in (0.75, 1.0, 1.25)]
        assert nu[0] > nu[1] > nu[2] > 1.0, (Ra, nu)
        assert et[0] > et[1] > et[2], (Ra, et)
        if Ra == 1e3:
            assert be[0] < be[1] < be[2], (Ra, be)


def test_heat_transfer_rises_and_bejan_falls_with_ra(steady):
    for n in (0.75, 1.0, 1.25):
        lo, hi = steady[(1e3, n)], steady[(1e4, n)]
        assert hi["Nu_hot_mean"] > lo["Nu_hot_mean"] and hi["E_total"] > lo["E_total"], n
        assert hi["Be"] < lo["Be"], n
        for d in (lo, hi):   # hot and cold walls carry the same heat at steady state
            assert abs(d["Nu_hot_mean"] - d["Nu_cold_mean"]) < 1e-3 * d["Nu_hot_mean"]


def test_total_entropy_near_table3(steady):
    """E_total of the 15^3 cavities lies within 10 % of Table 3's 51^3 values (7.4 % at most
    measured). Near conduction Table 3 sits about 4 % above the exact value 1, which is
    consistent with a factor (N/(N-1))^2 = 1.0404 in the paper's integral; the rest of the gap
    is the coarse grid."""
    for (Ra, n), d in steady.items():
        ref = TABLE3[(Ra, n)]
        assert abs(d["E_total"] / ref - 1.0) < 0.10, (Ra, n, d["E_total"], ref)


def test_newtonian_bejan_near_table4(steady):
    """For n = 1, where the viscosity in E_FF is 1 and the friction term has no reading to
    choose, Be of the 15^3 cavities lies within 0.05 of Table 4's 51^3 values (0.976 against
    0.975 at Ra = 1e3, 0.699 against 0.672 at Ra = 1e4)."""
    for Ra in (1e3, 1e4):
        assert abs(steady[(Ra, 1.0)]["Be"] - TABLE4[(Ra, 1.0)]) < 0.05, Ra

