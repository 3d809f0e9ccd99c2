"""Every stored reference minimum (tests/golden/fstar_<workload>_s<seed>.json) belongs to the
inputs that the seeded generator and the oracle's projector make today: the sinogram's sum and
sum of squares recorded with f* are reproduced (a change to the phantom recipe, the noise draw
order or the oracle's projector would otherwise leave the tests and the benchmark measuring
gaps against the minimum of another problem)."""
import glob
import json
import os

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
FILES = sorted(glob.glob(os.path.join(ROOT, "tests", "golden", "fstar_*_s*.json")))


def regenerate_b(workload, seed):
    import synth
    from oracle import fstar
    W = synth.WORKLOADS[workload]
    if W.get("geometry") == "cone":
        from oracle import cone as oc
        N, Nz, na, nr, nd, R = W["N"], W["Nz"], W["n_angles"], W["n_rows"], W["n_det"], W["src_dist"]
        g = oc.ConeGeometry(N, Nz, na, nr, nd, R, synth.fan_pitch(N, R, nd, W["cover"]),
                            synth.cone_row_pitch(N, Nz, R, nr, W["cover"]))
        return synth.ct3d_problem(seed, N, Nz, na, nr, nd, W["n_ellipses"], W["noise_frac"],
                                  lambda x: oc.K(x, g))["b"].astype(np.float64)
    P, _ = fstar.problem(workload, seed)
    return P.b


@pytest.mark.parametrize("path", FILES, ids=[os.path.basename(f) for f in FILES])
def test_golden_minimum_matches_regenerated_inputs(path):
    with open(path) as fh:
        gold = json.load(fh)
    if "b_sum" not in gold:
        pytest.skip("no fingerprint stored")
    b = regenerate_b(gold["workload"], gold["seed"])
    assert float(b.sum()) == pytest.approx(gold["b_sum"], rel=1e-12)
    assert float((b * b).sum()) == pytest.approx(gold["b_sumsq"], rel=1e-12)
