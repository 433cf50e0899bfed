"""Mass preconditioning and nested integration on the device against the
oracle's trajectories (FP64 path), and the mixed path against the FP64 path."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1212_0785_gb300 import lqcd

pytestmark = pytest.mark.gpu

DIMS = (4, 4, 4, 4)


def _run(Uh, params, seed, trajs):
    U = lqcd.gauge_field(DIMS).upload(Uh)
    st = lqcd.HmcState(U, seed=seed)
    infos = [st.trajectory(params) for _ in range(trajs)]
    out = U.download()
    st.close()
    return out, infos


CASES = [  # (integrator, kappa_h, gauge_substeps, heavy_inner, chrono)
    (lqcd.LEAPFROG, 0.12, 0, False, 0),
    (lqcd.OMELYAN, 0.12, 3, False, 0),
    (lqcd.LEAPFROG, 0.10, 2, True, 0),
    (lqcd.OMELYAN, 0.0, 4, False, 0),
    (lqcd.OMELYAN, 0.12, 2, True, 3),
]


@pytest.mark.parametrize("integ,kh,m,inner,chrono", CASES)
def test_trajectory_matches_oracle(integ, kh, m, inner, chrono):
    Uh = orc.gauge_start(DIMS, seed=1, eps=0.3)
    tau, nsteps = 0.5, 4
    params = lqcd.hmc_params(5.6, 0.156, tau, nsteps, integ, cg=lqcd.cg_params(tol=1e-11), hasenbusch_kappa=kh,
                             gauge_substeps=m, heavy_inner=inner, chrono=chrono)
    Ug, infos = _run(Uh, params, 1, 2)
    Uo = Uh
    for traj, g in enumerate(infos):
        Uo, o = orc.hmc_trajectory_hb(DIMS, Uo, 5.6, 0.156, kh, tau, nsteps, integrator=integ, gauge_substeps=m,
                                      heavy_inner=inner, seed=1, traj=traj, cg_tol=1e-11)
        assert abs(g["dH"] - o["dH"]) < 1e-7, (traj, g["dH"], o["dH"])
        assert abs(g["H0"] - o["H0"]) < 1e-9 * abs(o["H0"])
        assert g["accepted"] == o["accepted"]
        assert g["cg_failures"] == 0
    assert np.max(np.abs(Ug - Uo)) < 1e-9


def test_solve_counts_of_preconditioning_and_nesting():
    """the inner level adds gauge-force evaluations, not solves; mass
    preconditioning solves for both pseudofermions at every outer kick"""
    Uh = orc.gauge_start(DIMS, seed=2, eps=0.3)
    cg = lqcd.cg_params(tol=1e-11)
    _, (g0,) = _run(Uh, lqcd.hmc_params(5.6, 0.156, 0.5, 4, lqcd.OMELYAN, cg=cg), 2, 1)
    _, (g1,) = _run(Uh, lqcd.hmc_params(5.6, 0.156, 0.5, 4, lqcd.OMELYAN, cg=cg, gauge_substeps=3), 2, 1)
    _, (g2,) = _run(Uh, lqcd.hmc_params(5.6, 0.156, 0.5, 4, lqcd.OMELYAN, cg=cg, hasenbusch_kappa=0.12), 2, 1)
    kicks = 2 * 4 + 1  # Omelyan, 4 steps, adjacent kicks merged
    assert g0["n_solves"] == kicks + 1  # and the action at the end
    assert g1["n_solves"] == g0["n_solves"]  # the fermion force stays on the outer level
    assert g2["n_solves"] == 2 * kicks + 1 + 2  # two pseudofermions, the refresh solve, two actions


@pytest.mark.parametrize("m,inner", [(0, False), (2, True)])
def test_mixed_precision_hasenbusch_close_to_fp64(m, inner):
    Uh = orc.gauge_start(DIMS, seed=3, eps=0.3)
    base = dict(beta=5.6, kappa=0.156, tau=0.5, nsteps=4, integrator=lqcd.OMELYAN, hasenbusch_kappa=0.12,
                gauge_substeps=m, heavy_inner=inner, chrono=3)
    U64, (g64,) = _run(Uh, lqcd.hmc_params(**base, cg=lqcd.cg_params(tol=1e-12)), 3, 1)
    Umx, (gmx,) = _run(Uh, lqcd.hmc_params(**base, cg=lqcd.cg_params(tol=1e-12, sloppy=lqcd.F16N, delta=0.01),
                                            force_prec=lqcd.F32), 3, 1)
    assert abs(gmx["dH"] - g64["dH"]) < 1e-3, (gmx["dH"], g64["dH"])
    assert np.max(np.abs(Umx - U64)) < 1e-5
    assert gmx["cg_true_rel_res_max"] <= 1e-12 and gmx["cg_failures"] == 0


def test_rejects_bad_hasenbusch_parameters():
    U = lqcd.gauge_field(DIMS).upload(orc.gauge_start(DIMS, seed=1, eps=0.3))
    st = lqcd.HmcState(U, seed=1)
    for bad in (dict(hasenbusch_kappa=0.2), dict(hasenbusch_kappa=-0.1), dict(gauge_substeps=-1)):
        with pytest.raises(lqcd.LqcdError):
            st.trajectory(lqcd.hmc_params(5.6, 0.156, 0.5, 2, **bad))
    st.close()
