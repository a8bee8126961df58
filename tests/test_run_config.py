"""Configuration handling of the run driver (paper_1312_1789_b300.run), on the
CPU: defaults, rejected keys and values, output times on dt_max multiples."""
import pytest

from paper_1312_1789_b300 import run


def test_defaults_and_overrides():
    c = run.load_config({"workload": "plummer1k", "t_end": 0.25, "dt_out": 0.0625})
    assert c["precision"] == "mixed" and c["graph_cycles"] == 64
    w = run.build_workload(c)
    assert w.n == 1024 and w.t_end == 0.25 and w.order == 6
    assert run._steps(c, w) == [0.0625, 0.125, 0.1875, 0.25]
    c = run.load_config({"workload": {"model": "plummer", "n": 300, "seed": 5}, "order": 8, "dt_max": 0.03125})
    w = run.build_workload(c)
    assert w.n == 300 and w.order == 8 and w.dt_max == 0.03125
    assert run._steps(c, w) == [w.t_end]


@pytest.mark.parametrize("cfg", [{"bogus": 1}, {"workload": "galaxy"}, {"precision": "fp16"}, {"order": 5},
                                 {"workload": {"model": "king", "n": 10}}])
def test_rejected_configurations(cfg):
    with pytest.raises(ValueError):
        run.load_config(cfg)


@pytest.mark.parametrize("t_end,dt_out", [(0.1, 0.1), (0.125, 0.03), (0.25, 0.1875)])
def test_output_times_must_synchronise_every_particle(t_end, dt_out):
    c = run.load_config({"t_end": t_end, "dt_out": dt_out})
    w = run.build_workload(c)
    with pytest.raises(ValueError):
        run._steps(c, w)


def test_ensemble_configuration_rules():
    ens = {"model": "ensemble", "clusters": 4, "lo": 256, "hi": 512}
    run.load_config({"workload": ens})
    for extra in ({"checkpoint": "x"}, {"resume": "x"}, {"autotune": 2}, {"order": 8}):
        with pytest.raises(ValueError):
            run.load_config(dict({"workload": ens}, **extra))
