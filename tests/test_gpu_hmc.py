"""GPU parity of the whole trajectory against the oracle: dH to 1e-8, identical
accept decisions, plaquette; and device-side reversibility and dH ~ dt^2."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1212_0785_gb300 import lqcd

pytestmark = pytest.mark.gpu

DIMS = (4, 4, 4, 4)  # the 4^4 workload: seed 1, eps 0.3, beta 5.6, kappa 0.156


def _run_gpu(Uh, params, seed, trajs):
    U = lqcd.gauge_field(DIMS).upload(Uh)
    st = lqcd.HmcState(U, seed=seed)
    infos = [st.trajectory(params) for _ in range(trajs)]
    out = U.download()
    st.close()
    return out, infos


@pytest.mark.parametrize("integrator,tau,nsteps", [(lqcd.LEAPFROG, 1.0, 10), (lqcd.OMELYAN, 0.2, 10),
                                                   (lqcd.LEAPFROG, 0.3, 6)])
def test_trajectory_matches_oracle(integrator, tau, nsteps):
    Uh = orc.gauge_start(DIMS, seed=1, eps=0.3)
    params = lqcd.hmc_params(5.6, 0.156, tau, nsteps, integrator, cg=lqcd.cg_params(tol=1e-10))
    Ug, infos = _run_gpu(Uh, params, 1, 2)
    Uo = Uh
    for traj, g in enumerate(infos):
        Uo, o = orc.hmc_trajectory(DIMS, Uo, 5.6, 0.156, tau, nsteps, integrator=integrator, seed=1, traj=traj,
                                   cg_tol=1e-10)
        assert abs(g["dH"] - o["dH"]) < 1e-8, (g["dH"], o["dH"])
        assert abs(g["H0"] - o["H0"]) < 1e-8 * abs(o["H0"])
        assert g["u"] == o["u"]
        marginal = abs(o["u"] - np.exp(-o["dH"])) < 1e-8
        assert marginal or g["accepted"] == int(o["accepted"])
        assert g["n_solves"] == o["n_solves"] and g["cg_failures"] == 0
        assert abs(g["cg_iters"] - o["cg_iters"]) <= o["n_solves"]
        assert abs(g["plaq"] - o["plaq"]) < 1e-10
    assert np.max(np.abs(Ug - Uo)) < 1e-9


def test_pure_gauge_trajectory_matches_oracle():
    Uh = orc.gauge_start(DIMS, seed=1, eps=0.3)
    params = lqcd.hmc_params(5.6, 0.0, 0.5, 8, lqcd.OMELYAN, n_flavors=0)
    Ug, (g,) = _run_gpu(Uh, params, 4, 1)
    Uo, o = orc.hmc_trajectory(DIMS, Uh, 5.6, 0.0, 0.5, 8, integrator=orc.OMELYAN, n_flavors=0, seed=4, traj=0)
    assert abs(g["dH"] - o["dH"]) < 1e-9 and g["accepted"] == int(o["accepted"])
    assert np.max(np.abs(Ug - Uo)) < 1e-11


def test_mixed_trajectory_close_to_fp64():
    Uh = orc.gauge_start(DIMS, seed=1, eps=0.3)
    base = dict(beta=5.6, kappa=0.156, tau=0.2, nsteps=10, integrator=lqcd.OMELYAN)
    _, (g64,) = _run_gpu(Uh, lqcd.hmc_params(**base, cg=lqcd.cg_params(tol=1e-10)), 1, 1)
    for sl in (lqcd.F32, lqcd.F16N, lqcd.BF16):
        _, (gm,) = _run_gpu(Uh, lqcd.hmc_params(**base, cg=lqcd.cg_params(tol=1e-10, sloppy=sl)), 1, 1)
        assert abs(gm["dH"] - g64["dH"]) < 1e-6, (sl, gm["dH"], g64["dH"])
        assert gm["cg_true_rel_res_max"] <= 1e-10


def test_reversibility_on_device():
    Uh = orc.gauge_start(DIMS, seed=1, eps=0.3)
    U = lqcd.gauge_field(DIMS).upload(Uh)
    st = lqcd.HmcState(U, seed=1)
    params = lqcd.hmc_params(5.6, 0.156, 0.3, 3, lqcd.OMELYAN, cg=lqcd.cg_params(tol=1e-13))
    st.refresh(params)
    _, P, _ = st.fields()
    P0 = P.download()
    for _ in range(3):
        st.md_step(params)
    assert np.abs(U.download() - Uh).max() > 1e-2
    P.upload(-P.download())
    for _ in range(3):
        st.md_step(params)
    assert np.abs(U.download() - Uh).max() < 1e-10
    assert np.abs(P.download() + P0).max() < 1e-10
    st.close()


def test_energy_conservation_dt_squared():
    Uh = orc.gauge_start(DIMS, seed=1, eps=0.3)
    dH = []
    for n in (5, 10):
        params = lqcd.hmc_params(5.6, 0.156, 0.25, n, lqcd.LEAPFROG, cg=lqcd.cg_params(tol=1e-12), metropolis=False)
        _, (g,) = _run_gpu(Uh, params, 1, 1)
        dH.append(g["dH"])
    assert 3.5 < dH[0] / dH[1] < 4.5


def test_mixed_trajectory_fp32_forces_close_to_fp64():
    """The benchmark's mixed configuration (FP16+norm solver, FP32 forces)
    against the FP64 GPU trajectory from the same start and momenta."""
    Uh = orc.gauge_start(DIMS, seed=1, eps=0.3)
    base = dict(beta=5.6, kappa=0.156, tau=0.2, nsteps=10, integrator=lqcd.OMELYAN)
    U64, (g64,) = _run_gpu(Uh, lqcd.hmc_params(**base, cg=lqcd.cg_params(tol=1e-10)), 1, 1)
    Um, (gm,) = _run_gpu(Uh, lqcd.hmc_params(**base, cg=lqcd.cg_params(tol=1e-10, sloppy=lqcd.F16N, delta=0.003),
                                             force_prec=lqcd.F32), 1, 1)
    assert abs(gm["dH"] - g64["dH"]) < 1e-4, (gm["dH"], g64["dH"])
    assert gm["accepted"] == g64["accepted"] == 1
    assert np.max(np.abs(Um - U64)) < 1e-5
    assert gm["cg_true_rel_res_max"] <= 1e-10


@pytest.mark.parametrize("sloppy", [lqcd.F64, lqcd.F16N])
def test_chronological_guess_trajectory(sloppy):
    """solves after the first of a trajectory start from the previous solution:
    the same trajectory to the solver tolerance, fewer CG iterations, and the
    final Hamiltonian solve starts converged"""
    Uh = orc.gauge_start(DIMS, seed=1, eps=0.3)
    cg = lqcd.cg_params(tol=1e-12, sloppy=sloppy, delta=0.01)
    base = dict(beta=5.6, kappa=0.156, tau=0.5, nsteps=8, integrator=lqcd.OMELYAN, cg=cg)
    U0, (g0,) = _run_gpu(Uh, lqcd.hmc_params(**base), 1, 1)
    U1, (g1,) = _run_gpu(Uh, lqcd.hmc_params(**base, chrono=True), 1, 1)
    assert abs(g1["dH"] - g0["dH"]) < 1e-7, (g1["dH"], g0["dH"])
    assert np.max(np.abs(U1 - U0)) < 1e-9
    assert g1["cg_iters"] < 0.85 * g0["cg_iters"], (g1["cg_iters"], g0["cg_iters"])
    assert g1["n_solves"] == g0["n_solves"] == 18 and g1["cg_true_rel_res_max"] <= 1e-12


@pytest.mark.parametrize("order", [2, 3, 4])
def test_extrapolated_guess_trajectory(order):
    """chrono k >= 2 starts each solve from the extrapolation through the last
    k solutions: the same trajectory to the solver tolerance, fewer iterations
    than the previous-solution guess, every solve within tolerance"""
    Uh = orc.gauge_start(DIMS, seed=1, eps=0.3)
    cg = lqcd.cg_params(tol=1e-12, sloppy=lqcd.F16N, delta=0.01)
    base = dict(beta=5.6, kappa=0.156, tau=0.5, nsteps=8, integrator=lqcd.OMELYAN, cg=cg)
    U0, (g0,) = _run_gpu(Uh, lqcd.hmc_params(**base), 1, 1)
    U1, (g1,) = _run_gpu(Uh, lqcd.hmc_params(**base, chrono=1), 1, 1)
    Uk, (gk,) = _run_gpu(Uh, lqcd.hmc_params(**base, chrono=order), 1, 1)
    assert abs(gk["dH"] - g0["dH"]) < 1e-7, (gk["dH"], g0["dH"])
    assert np.max(np.abs(Uk - U0)) < 1e-9
    assert gk["cg_iters"] < g1["cg_iters"], (gk["cg_iters"], g1["cg_iters"])
    assert gk["n_solves"] == 18 and gk["cg_true_rel_res_max"] <= 1e-12 and gk["cg_failures"] == 0


def test_extrapolated_guess_md_steps_and_leapfrog():
    """separate md_step calls (two solves at the same links between steps) and
    the leapfrog spacing give the same trajectory as the zero guess"""
    Uh = orc.gauge_start(DIMS, seed=2, eps=0.3)
    cg = lqcd.cg_params(tol=1e-12, sloppy=lqcd.F16N, delta=0.01)
    for integ in (lqcd.LEAPFROG, lqcd.OMELYAN):
        out = []
        for k in (0, 3):
            p = lqcd.hmc_params(5.6, 0.156, 0.5, 4, integ, cg=cg, chrono=k)
            U = lqcd.gauge_field(DIMS).upload(Uh)
            st = lqcd.HmcState(U, seed=4, chain=0)
            st.refresh(p)
            for _ in range(4):
                st.md_step(p)
            out.append((U.download(), st.hamiltonian(p)))
            st.close()
        assert np.max(np.abs(out[1][0] - out[0][0])) < 1e-9
        assert abs(out[1][1] - out[0][1]) < 1e-7


def test_mixed_hamiltonian_plaquette_from_float_float_links():
    """with the mixed solver the Hamiltonians take the plaquette from the
    float-float link copy: H0 and H after MD steps agree with the FP64 path's"""
    Uh = orc.gauge_start((6, 4, 4, 8), seed=9, eps=0.4)
    cg64 = lqcd.cg_params(tol=1e-12)
    cgmx = lqcd.cg_params(tol=1e-12, sloppy=lqcd.F16N, delta=0.01)
    out = []
    for cg in (cg64, cgmx):
        U = lqcd.gauge_field((6, 4, 4, 8)).upload(Uh)
        st = lqcd.HmcState(U, seed=9)
        p = lqcd.hmc_params(5.7, 0.15, 0.4, 2, lqcd.LEAPFROG, cg=cg)
        h0 = st.refresh(p)
        st.md_step(p)
        out.append((h0, st.hamiltonian(p)))
        st.close()
    assert abs(out[1][0] - out[0][0]) < 1e-10 * abs(out[0][0])
    assert abs(out[1][1] - out[0][1]) < 1e-6 * abs(out[0][1])


@pytest.mark.parametrize("force_prec", [lqcd.F64, lqcd.F32])
def test_minimal_residual_guess_trajectory(force_prec):
    """chrono 3 with the minimal residual refinement (paper Sec. 6.2): the
    same trajectory as the zero guess to the solver tolerance (FP64 forces),
    or to the FP32 rounding of the solution (FP32 forces); every solve with
    two earlier solutions at distinct times refines its guess; fewer
    iterations than the zero guess"""
    Uh = orc.gauge_start(DIMS, seed=1, eps=0.3)
    cg = lqcd.cg_params(tol=1e-12, sloppy=lqcd.F16N, delta=0.01)
    base = dict(beta=5.6, kappa=0.156, tau=0.5, nsteps=8, integrator=lqcd.OMELYAN, cg=cg, force_prec=force_prec)
    U0, (g0,) = _run_gpu(Uh, lqcd.hmc_params(**base), 1, 1)
    Uk, (gk,) = _run_gpu(Uh, lqcd.hmc_params(**base, chrono=3), 1, 1)
    Um, (gm,) = _run_gpu(Uh, lqcd.hmc_params(**base, chrono=3, chrono_mre=True), 1, 1)
    print("iterations: zero guess", g0["cg_iters"], "extrapolated", gk["cg_iters"], "minimal residual",
          gm["cg_iters"], "refined", gm["cg_guesses_refined"], "accurate residuals", gk["cg_accurate_residuals"],
          gm["cg_accurate_residuals"])
    tol_dh, tol_u = (1e-7, 1e-9) if force_prec == lqcd.F64 else (1e-5, 1e-6)
    assert abs(gm["dH"] - g0["dH"]) < tol_dh, (gm["dH"], g0["dH"])
    assert np.max(np.abs(Um - U0)) < tol_u
    # 17 force evaluations and the final action: solves 3..17 have two earlier solutions
    assert gm["cg_guesses_refined"] == 15 and gk["cg_guesses_refined"] == 0
    assert gm["cg_iters"] < g0["cg_iters"]
    assert gm["n_solves"] == 18 and gm["cg_true_rel_res_max"] <= 1e-12 and gm["cg_failures"] == 0
