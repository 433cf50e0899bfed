"""The benchmark's own mixed-precision configuration against the FP64 oracle,
result by result: FP16+norm solver storage with delta 0.003, FP32 forces and
FP32 exponential with the float-float link product, the chronological guess
extrapolated through the last 3 solutions, Omelyan 2MN with 16 steps, tau 1,
beta 5.8, kappa 0.1570, start exp(i 0.15 H) from Philox seed 3, CG true
|r|/|b| <= 1e-10 -- on 4^4 (two chained trajectories, Metropolis on) and 8^4
(one trajectory, Metropolis off so that the compared links are the evolved
ones).  One chain of a batch of chains is held to the same bar.

The tolerances follow from the FP32 molecular dynamics.  A force evaluation rounds the links and the solution
to FP32 and adds in FP32, so each of the 32 V momentum coefficients is moved by
about 2^-24 |F| per evaluation, in no coherent direction; over tau = 1 with
|F| ~ 1-3 and |P| ~ 1 that changes H1 by about 2e-7 sqrt(32 V), and every link
entry by a few 1e-7 (with 2 nsteps FP32 exponentials of error ~1e-7 each).
The bounds sit 5-50 times above those estimates (measured: dH 1.4e-5 at 4^4,
1.6e-5 at 8^4; links 2.6e-7; X 1.2e-7; plaquette 1.3e-9).  A dropped or
mis-signed term anywhere changes dH by O(1).  The first trajectory starts from
bitwise the oracle's links, so H0 and phi agree to FP64 rounding; a chained
trajectory starts from links that already differ by the previous trajectory's
link error dU, which moves S_g by at most 24 beta V dU.
"""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1212_0785_gb300 import lqcd
from tests.gpu_util import half

pytestmark = pytest.mark.gpu

BETA, KAPPA, TAU, NSTEPS, SEED, EPS = 5.8, 0.1570, 1.0, 16, 3, 0.15
TOL_H0_REL = 1e-12      # first trajectory: FP64 refresh (plaquette from float-float links, ~1e-14)
TOL_PHI_REL = 1e-12     # phi = Mhat^dag eta in FP64, on the trajectory's start links
TOL_LINKS = 1e-5        # max |U_gpu - U_oracle| over all link entries
TOL_PLAQ = 1e-8         # mean plaquette after the trajectory
TOL_X_REL = 1e-5        # max |X_gpu - X_oracle| / max |X_oracle| of the final solve


def tol_dh(dims):
    """|dH_gpu - dH_oracle| <= 1e-6 sqrt(32 V): 9.1e-5 at 4^4, 3.6e-4 at 8^4"""
    return 1e-6 * np.sqrt(32 * int(np.prod(dims)))


def tol_h0_rel(dims, H0, dU_prev):
    """relative H0 bound of a trajectory whose start links differ from the
    oracle's by dU_prev (0 for the first trajectory)"""
    return TOL_H0_REL + 24 * BETA * int(np.prod(dims)) * dU_prev / abs(H0)


def bench_params(metropolis=True, mre=False):
    cg = lqcd.cg_params(tol=1e-10, maxiter=20000, sloppy=lqcd.F16N, delta=0.003)
    return lqcd.hmc_params(BETA, KAPPA, TAU, NSTEPS, lqcd.OMELYAN, n_flavors=2, cg=cg, force_prec=lqcd.F32,
                           chrono=3, metropolis=metropolis, chrono_mre=mre)


def final_solution_error(dims, U_gpu, phi_gpu, U_or, phi_or):
    """X = (Mhat^dag Mhat)^-1 phi on the trajectory's final links: the GPU's
    mixed solver on the GPU's links against the oracle's CG on the oracle's"""
    x = lqcd.spinor_field(dims, 0)
    Us = lqcd.gauge_field(dims, lqcd.F16N).copy_from(U_gpu)
    rc, info = lqcd.cg_solve(x, U_gpu, phi_gpu, KAPPA,
                             lqcd.cg_params(tol=1e-10, maxiter=20000, sloppy=lqcd.F16N, delta=0.003), U_sloppy=Us)
    assert rc == lqcd.OK and info.true_rel_res <= 1e-10
    xo, conv, _, _ = orc.cg(dims, U_or, KAPPA, phi_or, tol=1e-10)
    assert conv
    xo = half(xo, dims, 0)
    return float(np.max(np.abs(x.download() - xo)) / np.max(np.abs(xo)))


def run_and_compare(dims, trajs, metropolis, mre=False):
    """the GPU chain and the oracle chain from the same start, trajectory by
    trajectory; returns the list of per-result errors"""
    p = bench_params(metropolis, mre)
    U = lqcd.gauge_field(dims)
    lqcd.gauge_start(U, SEED, EPS)
    st = lqcd.HmcState(U, seed=SEED)
    _, _, phi = st.fields()
    Uo = orc.gauge_start(dims, SEED, EPS)
    assert np.max(np.abs(U.download() - Uo)) < 1e-13
    errs = []
    dU_prev = 0.0
    for traj in range(trajs):
        Uo_start = Uo
        g = st.trajectory(p)
        Uo, o = orc.hmc_trajectory(dims, Uo_start, BETA, KAPPA, TAU, NSTEPS, integrator=orc.OMELYAN, seed=SEED,
                                   traj=traj, cg_tol=1e-10, metropolis=metropolis)
        phi_or = orc.mhat(dims, Uo_start, KAPPA, orc.eta_refresh(dims, SEED, traj), dagger=True)
        e = {"dH": abs(g["dH"] - o["dH"]), "H0_rel": abs(g["H0"] - o["H0"]) / abs(o["H0"]),
             "plaq": abs(g["plaq"] - o["plaq"]), "links": float(np.max(np.abs(U.download() - Uo))),
             "phi_rel": float(np.max(np.abs(phi.download() - half(phi_or, dims, 0))) / np.max(np.abs(phi_or))),
             "accept": (g["accepted"], int(o["accepted"])), "u": (g["u"], o["u"]), "dH_oracle": o["dH"],
             "H0_tol": tol_h0_rel(dims, o["H0"], dU_prev), "phi_tol": TOL_PHI_REL + 10 * dU_prev}
        e["X_rel"] = final_solution_error(dims, U, phi, Uo, phi_or)
        dU_prev = e["links"]
        errs.append(e)
        print(dims, traj, e)
        assert g["cg_true_rel_res_max"] <= 1e-10 and g["cg_failures"] == 0
        assert g["n_solves"] == o["n_solves"]
    st.close()
    return errs


def check(dims, errs):
    for e in errs:
        assert e["u"][0] == e["u"][1]
        marginal = abs(e["u"][1] - np.exp(-e["dH_oracle"])) < tol_dh(dims)
        assert marginal or e["accept"][0] == e["accept"][1], e
        assert e["H0_rel"] < e["H0_tol"], e
        assert e["phi_rel"] < e["phi_tol"], e
        assert e["dH"] < tol_dh(dims), e
        assert e["plaq"] < TOL_PLAQ, e
        assert e["links"] < TOL_LINKS, e
        assert e["X_rel"] < TOL_X_REL, e


@pytest.mark.parametrize("mre", [False, True])
def test_benchmark_configuration_matches_oracle_4x4x4x4(mre):
    """(with mre: the guesses refined by minimal residual extrapolation)"""
    dims = (4, 4, 4, 4)
    errs = run_and_compare(dims, 2, metropolis=True, mre=mre)
    assert errs[0]["accept"] == (1, 1)  # dH 0.35 against u 0.082: the compared links moved
    check(dims, errs)


def test_benchmark_configuration_matches_oracle_8x8x8x8():
    dims = (8, 8, 8, 8)
    errs = run_and_compare(dims, 1, metropolis=False)
    check(dims, errs)


def test_batched_chain_matches_oracle():
    """three chains of the batched-chains recipe (leapfrog 10 steps, tau 1,
    start eps 0.3, FP16+norm solver, FP32 forces, chrono 3) advanced as one
    batch; the 4^4 and 6x4x2x10 chains each against the oracle"""
    specs = [((4, 4, 4, 4), 5.6, 0.150, 100), ((6, 4, 2, 10), 5.75, 0.1535, 101), ((8, 6, 6, 12), 5.9, 0.157, 102)]
    cg = lqcd.cg_params(tol=1e-10, maxiter=20000, sloppy=lqcd.F16N, delta=0.003)
    params = [lqcd.hmc_params(b, k, 1.0, 10, lqcd.LEAPFROG, cg=cg, force_prec=lqcd.F32, chrono=3,
                              metropolis=False) for _, b, k, _ in specs]
    fields, states = [], []
    for i, (dims, _, _, seed) in enumerate(specs):
        U = lqcd.gauge_field(dims)
        lqcd.gauge_start(U, seed, 0.3)
        fields.append(U)
        states.append(lqcd.HmcState(U, seed=seed, chain=i))
    batch = lqcd.Batch(states)
    got = batch.trajectory(params)
    for i, (dims, beta, kappa, seed) in enumerate(specs[:2]):
        Uo, o = orc.hmc_trajectory(dims, orc.gauge_start(dims, seed, 0.3), beta, kappa, 1.0, 10,
                                   integrator=orc.LEAPFROG, seed=seed, chain=i, traj=0, cg_tol=1e-10,
                                   metropolis=False)
        g = got[i]
        print(dims, g["dH"], o["dH"], np.max(np.abs(fields[i].download() - Uo)))
        assert abs(g["dH"] - o["dH"]) < tol_dh(dims)
        assert abs(g["H0"] - o["H0"]) < TOL_H0_REL * abs(o["H0"])
        assert abs(g["plaq"] - o["plaq"]) < TOL_PLAQ
        assert np.max(np.abs(fields[i].download() - Uo)) < TOL_LINKS
        assert g["u"] == o["u"] and g["n_solves"] == o["n_solves"] and g["cg_true_rel_res_max"] <= 1e-10
    batch.close()
    for st in states:
        st.close()
