"""The run driver (paper_1312_1789_b300.run) on the GPU: outputs at dt_max
multiples with small energy and momentum drift, checkpoints at each output,
and a run resumed from a checkpoint that ends in the same state, bit for bit,
as the uninterrupted one."""
import io
import json
import os

import numpy as np
import pytest

from paper_1312_1789_b300 import run

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,cycles", [("mixed", 8), ("fp64", 0)])
def test_run_outputs_checkpoints_and_bitwise_resume(tmp_path, precision, cycles):
    cfg = {"workload": {"model": "plummer", "n": 700, "seed": 12, "eps": 1e-3}, "precision": precision,
           "t_end": 0.25, "dt_out": 0.0625, "graph_cycles": cycles, "checkpoint": str(tmp_path / "ck" / "a")}
    log = io.StringIO()
    recs = run.run(cfg, log)
    assert [r["t"] for r in recs] == [0.0625, 0.125, 0.1875, 0.25]
    assert [json.loads(l)["t"] for l in log.getvalue().splitlines()] == [r["t"] for r in recs]
    for r in recs:
        assert abs(r["dE_E"]) < 1e-4 and r["dP_rel"] < 1e-5
        assert sum(r["nact_histogram"].values()) > 0
    assert recs[-1]["blocks"] == sum(sum(r["nact_histogram"].values()) for r in recs)
    full = np.load(tmp_path / "ck" / "a_last.npz")
    # resume from the second output: the same end state and counts
    cfg2 = dict(cfg, checkpoint=str(tmp_path / "b"), resume=str(tmp_path / "ck" / "a_t0.125.npz"))
    recs2 = run.run(cfg2)
    assert [r["t"] for r in recs2] == [0.1875, 0.25]
    assert recs2[-1]["blocks"] == recs[-1]["blocks"] and recs2[-1]["interactions"] == recs[-1]["interactions"]
    resumed = np.load(tmp_path / "b_last.npz")
    for key in ("x", "v", "d", "t", "dt"):
        assert np.array_equal(resumed[key], full[key]), key
    assert recs2[-1]["dE_E"] == recs[-1]["dE_E"]
    # a checkpoint of another workload is refused
    with pytest.raises(ValueError):
        run.run(dict(cfg, workload={"model": "plummer", "n": 700, "seed": 13, "eps": 1e-3},
                     resume=str(tmp_path / "ck" / "a_last.npz"), checkpoint=None))


def test_ensemble_run_reports_per_cluster_energy_errors():
    cfg = {"workload": {"model": "ensemble", "clusters": 6, "lo": 256, "hi": 1024}, "t_end": 0.125,
           "dt_out": 0.0625, "graph_cycles": 8}
    recs = run.run(cfg)
    assert [r["t"] for r in recs] == [0.0625, 0.125]
    assert recs[-1]["cycles"] > recs[0]["cycles"] > 0
    assert 0 <= recs[-1]["dE_E_median"] <= recs[-1]["dE_E_worst"] < 1e-3
