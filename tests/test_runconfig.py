"""The bundled run configurations (no GPU): every one parses, builds the
population it describes, and maps onto Simulator options."""
import json

import pytest

from paper_2311_08927_gb300 import chad as CH
from paper_2311_08927_gb300 import runconfig as RC


@pytest.mark.parametrize("name,n,intervals,prec,learned", [
    ("c1", 1000, 1440, CH.PREC_FP64, 0), ("c2", 100_000, 14_400, CH.PREC_FP64, 0),
    ("c3", 1_000_000, 7200, CH.PREC_MIXED, 1), ("c4", 2_000_000, 7200, CH.PREC_MIXED, 1)])
def test_bundled_configs(name, n, intervals, prec, learned):
    cfg = RC.read(RC.path(name))
    assert cfg["particles"] == n
    pop, kw, dt, k = RC.load(RC.path(name), particles=500)
    assert pop.n == 500 and dt == 60.0 and k == intervals
    assert kw["precision"] == prec and kw["learned"] == learned and kw["rtol"] == 1e-6
    assert kw["h2_algebraic"]  # the paper's Eq. 8 model, as the benchmark runs it


def test_many_digester_config():
    pop, kw, dt, k = RC.load(RC.path("c5"), particles=3000)
    assert len(pop.digesters) == 64 and k == 2880 and kw["learned"] == 1
    assert all(d.flow is not None for d in pop.digesters)


def test_diffusion_and_bad_configs(tmp_path):
    good = {"name": "x", "workload": 2, "particles": 2000, "precision": "fp64",
            "h2_algebraic": True, "diffusion": {"D": 1e-6, "h": 0.006}, "intervals": 3}
    p = tmp_path / "x.json"
    p.write_text(json.dumps(good))
    pop, kw, dt, k = RC.load(str(p))
    assert kw["diffusion"] == (1e-6, 0.006) and kw["h2_algebraic"] and k == 3 and pop.n == 2000
    for bad in ({"workload": 9}, {"precision": "fp16"}, {"h2_algebraic": True, "precision": "mixed_f32rates"},
                {"typo": 1}, {"diffusion": {"D": 1e-6, "h": 0.0}}):
        q = tmp_path / "bad.json"
        q.write_text(json.dumps({**good, **bad}))
        with pytest.raises(ValueError):
            RC.read(str(q))
