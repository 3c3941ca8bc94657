"""Run configurations as JSON (``configs/c1.json`` .. ``c5.json``): the
workload recipe (``inputs.config_population``), the integrator form and
tolerances, the coupling interval and the number of intervals, and optional
diffusion between particles.  ``load`` turns one into a Population and the
keyword arguments of ``chad.Simulator``."""
from __future__ import annotations

import json
import os

from . import inputs as I

CONFIG_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "configs")
FORMS = {"fp64": 0, "mixed": 1, "mixed_f32rates": 2}
KEYS = {"name", "workload", "particles", "note", "precision", "learned", "h2_algebraic", "rtol",
        "coupling_interval_s", "intervals", "diffusion"}


def path(name: str) -> str:
    """The bundled configuration of that name (c1 .. c5)."""
    return os.path.join(CONFIG_DIR, f"{name}.json")


def read(p: str) -> dict:
    """Parse and check a run configuration; ValueError on an unknown key or value."""
    with open(p) as f:
        cfg = json.load(f)
    unknown = set(cfg) - KEYS
    if unknown:
        raise ValueError(f"unknown keys {sorted(unknown)} in {p}")
    if cfg.get("workload") not in (1, 2, 3, 4, 5):
        raise ValueError("workload must be 1 .. 5")
    if cfg.get("precision", "fp64") not in FORMS:
        raise ValueError(f"precision must be one of {sorted(FORMS)}")
    if cfg.get("h2_algebraic") and cfg.get("precision", "fp64") == "mixed_f32rates":
        raise ValueError("h2_algebraic takes the fp64 or the mixed form")
    if not cfg.get("rtol", 1e-6) > 0 or not cfg.get("coupling_interval_s", 60.0) > 0:
        raise ValueError("rtol and coupling_interval_s must be > 0")
    if int(cfg.get("intervals", 1)) < 0:
        raise ValueError("intervals must be >= 0")
    dif = cfg.get("diffusion")
    if dif is not None and not (dif.get("D", 0) >= 0 and dif.get("h", 0) > 0):
        raise ValueError("diffusion needs D >= 0 and h > 0")
    return cfg


def load(p: str, particles: int | None = None):
    """(Population, Simulator keyword arguments, coupling interval in s,
    intervals) of a run configuration; particles overrides its count."""
    cfg = read(p)
    n = particles if particles is not None else cfg.get("particles")
    pop = I.config_population(int(cfg["workload"]), n=n)
    kw = dict(precision=FORMS[cfg.get("precision", "fp64")], rtol=float(cfg.get("rtol", 1e-6)),
              learned=1 if cfg.get("learned") else 0,
              h2_algebraic=bool(cfg.get("h2_algebraic", False)))
    dif = cfg.get("diffusion")
    if dif is not None:
        kw["diffusion"] = (float(dif["D"]), float(dif["h"]))
    return pop, kw, float(cfg.get("coupling_interval_s", 60.0)), int(cfg.get("intervals", 1))
