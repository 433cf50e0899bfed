"""The threads-per-block autotuner (paper Sec. 4): every candidate of every
tunable kernel class is timed on a lattice and the fastest kept and written
out; launches on that lattice then use it.  The force and link-update kernels
give bitwise the same results at every block size, and so does the plain
hopping term (no block sums); a whole trajectory with the tuned table agrees
with the default one to the solver's tolerance."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1212_0785_gb300 import inputs, lqcd
from tests.gpu_util import half

pytestmark = pytest.mark.gpu


@pytest.fixture
def clean_table():
    lqcd.autotune_clear()
    yield
    lqcd.autotune_clear()


def test_autotune_writes_and_applies_the_table(tmp_path, clean_table):
    dims = (8, 8, 8, 8)
    path = tmp_path / "tune.txt"
    best = lqcd.autotune(dims, path)
    rows = lqcd.read_tune_table(path)
    for k in lqcd.TUNED_CLASSES:
        mine = [r for r in rows if r["class"] == k and r["dims"] == dims]
        assert len(mine) >= 3 and sum(r["best"] for r in mine) == 1
        fastest = min(mine, key=lambda r: r["ms"])
        assert best[k] == fastest["block"] == [r for r in mine if r["best"]][0]["block"]
        assert all(r["ms"] > 0 for r in mine)
    lqcd.autotune_clear()
    assert lqcd.autotune_block("gauge_force_f32", dims) == 0
    lqcd.autotune_load(path)
    assert {k: lqcd.autotune_block(k, dims) for k in lqcd.TUNED_CLASSES} == best


def _write(path, dims, blocks):
    with open(path, "w") as fh:
        for k, b in blocks.items():
            fh.write(f"{k} {dims[0]} {dims[1]} {dims[2]} {dims[3]} {b} 1.0 1\n")


@pytest.mark.parametrize("block", [32, 96, 256])
def test_force_and_link_update_bitwise_at_every_block_size(tmp_path, block, clean_table):
    dims = (6, 4, 2, 10)
    Uh = orc.gauge_start(dims, seed=5, eps=0.4)
    Ph = inputs.random_momentum(dims, 18)
    X = inputs.random_spinor(dims, 19, parity=0)
    out = {}
    for tag in ("default", "tuned"):
        if tag == "tuned":
            fb = min(block, 128)
            _write(tmp_path / "t.txt", dims, {"gauge_force_f32": block, "gauge_force_f64": block,
                                             "fermion_force_f32": fb, "link_update_f32": block})
            lqcd.autotune_load(tmp_path / "t.txt")
        U = lqcd.gauge_field(dims).upload(Uh)
        P = lqcd.momentum_field(dims).upload(Ph)
        x = lqcd.spinor_field(dims, 0).upload(half(X, dims, 0))
        lqcd.gauge_force(P, U, 5.6, 0.03, arith=lqcd.F32)
        lqcd.gauge_force(P, U, 5.6, 0.03)
        lqcd.fermion_force(P, U, x, 0.15, 0.02, arith=lqcd.F32)
        lqcd.link_update(U, P, 0.05, arith=lqcd.F32)
        out[tag] = (P.download(), U.download())
    assert np.array_equal(out["default"][0], out["tuned"][0])
    assert np.array_equal(out["default"][1], out["tuned"][1])


def test_hop_bitwise_at_every_block_size(tmp_path, clean_table):
    dims = (8, 6, 6, 12)  # Vh = 1728: ragged last blocks at 64, 128 and 256
    Uh = inputs.random_gauge(dims, 40, spread=0.5)
    U = lqcd.gauge_field(dims).upload(Uh)
    Us = lqcd.gauge_field(dims, lqcd.F16N).copy_from(U)
    psi = lqcd.spinor_field(dims, 0, lqcd.F16N).copy_from(
        lqcd.spinor_field(dims, 0).upload(half(inputs.random_spinor(dims, 41, parity=0), dims, 0)))
    outs = []
    for b in (64, 128, 256):
        _write(tmp_path / "h.txt", dims, {"dslash_f16n": b})
        lqcd.autotune_load(tmp_path / "h.txt")
        o = lqcd.spinor_field(dims, 1, lqcd.F16N)
        lqcd.dslash(o, Us, psi, True)
        outs.append(o.download())
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[1], outs[2])


def test_tuned_trajectory_matches_default(tmp_path, clean_table):
    dims = (4, 4, 4, 4)
    cg = lqcd.cg_params(tol=1e-12, sloppy=lqcd.F16N, delta=0.01)
    p = lqcd.hmc_params(5.6, 0.156, 0.5, 4, lqcd.OMELYAN, cg=cg, force_prec=lqcd.F32, chrono=3)
    res = []
    for tune in (False, True):
        if tune:
            lqcd.autotune(dims, tmp_path / "t4.txt")
        U = lqcd.gauge_field(dims)
        lqcd.gauge_start(U, 1, 0.3)
        st = lqcd.HmcState(U, seed=1)
        res.append((st.trajectory(p), U.download()))
        st.close()
    assert abs(res[0][0]["dH"] - res[1][0]["dH"]) < 1e-7
    assert np.max(np.abs(res[0][1] - res[1][1])) < 1e-9
