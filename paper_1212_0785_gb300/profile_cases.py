"""Small fixed workloads for profiling the library's kernels under ncu.

  python -m paper_1212_0785_gb300.profile_cases dslash   # 3 launches per precision
  python -m paper_1212_0785_gb300.profile_cases cg       # one mixed solve
  python -m paper_1212_0785_gb300.profile_cases md       # FP32 MD forces + FP32 link update
  python -m paper_1212_0785_gb300.profile_cases traj     # one 1-step mixed trajectory (the HMC's own kernels)

Each case builds the 32^3x64 start configuration of the benchmark (Philox
seed 3, eps 0.15) unless --dims is given, runs its calls once and exits 0.
They hold a few GB on the device at most, so a `--set full` capture of a
handful of their launches ends in a minute or two.
"""
from __future__ import annotations

import argparse
import sys

import torch

from . import lqcd

KAPPA, BETA = 0.1570, 5.8


def _start(dims):
    U = lqcd.gauge_field(dims)
    lqcd.gauge_start(U, seed=3, eps=0.15)
    eta = lqcd.spinor_field(dims, 0)
    lqcd.eta_refresh(eta, seed=3, traj=0)
    return U, eta


def case_dslash(dims):
    """three half hopping terms per storage precision: F16N, F32, BF16, F64"""
    U, eta = _start(dims)
    for prec in (lqcd.F16N, lqcd.F32, lqcd.BF16, lqcd.F64):
        Us = U if prec == lqcd.F64 else lqcd.gauge_field(dims, prec).copy_from(U)
        inp = eta if prec == lqcd.F64 else lqcd.spinor_field(dims, 0, prec).copy_from(eta)
        out = lqcd.spinor_field(dims, 1, prec)
        for _ in range(3):
            lqcd.dslash(out, Us, inp)
        torch.cuda.synchronize()


def case_cg(dims):
    """phi = Mhat^dag eta (two FP64 hopping terms), then the benchmark's mixed
    solve (FP16+norm, delta 0.003, tol 1e-10)"""
    U, eta = _start(dims)
    b = lqcd.spinor_field(dims, 0)
    lqcd.mhat(b, U, eta, KAPPA, True)
    x = lqcd.spinor_field(dims, 0)
    Us = lqcd.gauge_field(dims, lqcd.F16N).copy_from(U)
    rc, info = lqcd.cg_solve(x, U, b, KAPPA, lqcd.cg_params(tol=1e-10, sloppy=lqcd.F16N, delta=0.003), U_sloppy=Us)
    torch.cuda.synchronize()
    print(f"cg: status {rc}, {info.iters} iterations, {info.restarts} reliable updates, "
          f"true |r|/|b| {info.true_rel_res:.2e}")


def case_md(dims):
    """FP32 gauge force, FP32 fermion force and one FP32 link update (the
    molecular dynamics of the mixed trajectory)"""
    U, eta = _start(dims)
    P = lqcd.momentum_field(dims)
    lqcd.momentum_refresh(P, seed=3, traj=0)
    lqcd.gauge_force(P, U, BETA, 0.01, arith=lqcd.F32)
    lqcd.fermion_force(P, U, eta, KAPPA, 0.01, arith=lqcd.F32)
    lqcd.link_update(U, P, 0.03, arith=lqcd.F32)
    torch.cuda.synchronize()


def case_traj(dims):
    """one mixed-precision trajectory of one Omelyan step (the benchmark's
    settings otherwise): every kernel of the trajectory in the variants the
    HMC driver launches"""
    U = lqcd.gauge_field(dims)
    lqcd.gauge_start(U, seed=3, eps=0.15)
    st = lqcd.HmcState(U, seed=3)
    cg = lqcd.cg_params(tol=1e-10, maxiter=20000, sloppy=lqcd.F16N, delta=0.003)
    info = st.trajectory(lqcd.hmc_params(BETA, KAPPA, 1.0, 1, lqcd.OMELYAN, cg=cg, force_prec=lqcd.F32, chrono=3))
    torch.cuda.synchronize()
    print(f"traj: dH {info['dH']:.4f}, {info['cg_iters']} CG iterations, {info['n_solves']} solves")
    st.close()


CASES = {"dslash": case_dslash, "cg": case_cg, "md": case_md, "traj": case_traj}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("case", choices=sorted(CASES))
    ap.add_argument("--dims", type=int, nargs=4, default=(32, 32, 32, 64))
    args = ap.parse_args(argv)
    CASES[args.case](tuple(args.dims))
    return 0


if __name__ == "__main__":
    sys.exit(main())
