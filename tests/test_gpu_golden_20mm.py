"""The CUDA path on the full 20 x 10 x 4 mm plate (160 x 80 x 32 coarse
hexahedra, 129 x 129 x 65-node fine patch, m = 8) against the FP64 oracle's
fields stored in tests/golden/multitrack_20mm_oracle.npz (written by
tests/golden/make_multitrack_20mm.py, which runs only the oracle).

Bars: the plain FP64 path within 1e-9 relative L2 of the oracle on both
levels; the precision form (FP32 inner CG, FP64 defect correction to 1e-10)
within 1e-6; element states (the melt-pool mask included) bit-exact on both
levels, with no element mean within 1e-6 K of T_melt in the oracle's run."""
import os

import numpy as np
import pytest

from paper_2110_12932_gb300 import build as tlbuild
from paper_2110_12932_gb300 import tl, workloads

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "multitrack_20mm_oracle.npz")


@pytest.fixture(scope="module", autouse=True)
def lib():
    tlbuild.build()
    return tl.load()


def load_golden():
    z = np.load(GOLDEN)
    out = {}
    T0 = float(z["T0"])
    for n in (int(s) for s in z["steps"]):
        snap = {"origin": tuple(int(v) for v in z[f"s{n}_origin"])}
        for lvl in ("fine", "coarse"):
            T = np.full(int(z[f"s{n}_{lvl}_n"]), T0)
            T[z[f"s{n}_{lvl}_idx"]] = z[f"s{n}_{lvl}_val"]
            snap[lvl] = T
            snap[f"{lvl}_state"] = z[f"s{n}_{lvl}_state"]
        snap["tie_distance"] = z[f"s{n}_tie_distance"]
        out[n] = snap
    return out


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("precision,tol,bar", [(tl.TL_FP64, 1e-12, 1e-9), (tl.TL_FP32_REFINED, 1e-10, 1e-6)])
def test_20mm_plate_against_stored_oracle(precision, tol, bar):
    gold = load_golden()
    cfg = workloads.workload("multitrack_20mm", precision=precision, tol=tol, tol_inner=1e-5)
    prob = tl.Problem(cfg)
    done = 0
    for n in sorted(gold):
        prob.macro_steps(n - done)
        done = n
        g = gold[n]
        assert np.all(g["tie_distance"] > 1e-6), "threshold ties in the oracle's run"
        Tf, org = prob.temperature(tl.TL_FINE)
        Tc, _ = prob.temperature(tl.TL_COARSE)
        assert tuple(org) == g["origin"], (n, org, g["origin"])
        ef, ec = rel(Tf, g["fine"]), rel(Tc, g["coarse"])
        print(f"macro step {n}: fine rel L2 {ef:.3e}, coarse rel L2 {ec:.3e}")
        assert ef <= bar and ec <= bar, (n, ef, ec)
        sf, sc = prob.state(tl.TL_FINE), prob.state(tl.TL_COARSE)
        assert np.array_equal(sf, g["fine_state"]), (n, np.count_nonzero(sf != g["fine_state"]))
        assert np.array_equal(sc, g["coarse_state"]), (n, np.count_nonzero(sc != g["coarse_state"]))
        assert np.count_nonzero(sf == tl.MELTED) > 0, "the melt pool must be non-empty"
    prob.close()
