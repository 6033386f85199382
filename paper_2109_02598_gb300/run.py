"""A run from a configuration file (the paper's standardized problem parameters and data
persistence, Sec. 2.3.4-2.3.5).

    python -m paper_2109_02598_gb300.run config.json

The configuration is JSON:

    {"grid":  {"shape": [ny, nx] or [nz, ny, nx], "h": 1.0},
     "model": {"name": "ac" | "ch" | "gs" | "c", "coeffs": [...], "dt": 0.05,
               "stencil": "std"},                                   (stencil optional)
     "init":  {"checkpoint": "path.npz"}                            (resume a run), or
              {"npy": ["field0.npy", ...]}                          (float32 arrays), or
              {"synthetic": "cahn_hilliard_init", "args": {...}}    (the repository's
                                                                    seeded recipes),
     "run":   {"steps": 1000, "tuning": "auto" | [tx, ty, k] | null,
               "series_every": 100, "energy": false, "series_path": "series.json",
               "checkpoint_every": 0, "checkpoint_path": "ckpt_{step}.npz"}}

Every key of "run" but "steps" is optional. The runner writes the mass/energy series (and
the checkpoints) as it goes, and prints one JSON summary line at the end.
"""
from __future__ import annotations

import json
import os
import sys

import numpy as np

MODELS = {"ac": 1, "ch": 1, "gs": 2, "c": 2}


class ConfigError(ValueError):
    pass


def validate(cfg: dict) -> dict:
    """Check a configuration and fill in the defaults; raises ConfigError naming the problem."""
    if not isinstance(cfg, dict):
        raise ConfigError("the configuration must be a JSON object")
    for sect in ("grid", "model", "init", "run"):
        if not isinstance(cfg.get(sect), dict):
            raise ConfigError(f'missing section "{sect}"')
    g, m, i, r = cfg["grid"], cfg["model"], cfg["init"], cfg["run"]
    shape = g.get("shape")
    if (not isinstance(shape, list) or len(shape) not in (2, 3)
            or not all(isinstance(s, int) and s > 0 for s in shape)):
        raise ConfigError('"grid.shape" must be 2 or 3 positive integers')
    if m.get("name") not in MODELS:
        raise ConfigError(f'"model.name" must be one of {sorted(MODELS)}')
    if not isinstance(m.get("coeffs"), list) or not isinstance(m.get("dt"), (int, float)):
        raise ConfigError('"model" needs "coeffs" (a list) and "dt" (a number)')
    kinds = [k for k in ("checkpoint", "npy", "synthetic") if k in i]
    if len(kinds) != 1:
        raise ConfigError('"init" needs exactly one of "checkpoint", "npy", "synthetic"')
    if "npy" in i and (not isinstance(i["npy"], list) or len(i["npy"]) != MODELS[m["name"]]):
        raise ConfigError(f'"init.npy" must list {MODELS[m["name"]]} files for model '
                          f'"{m["name"]}"')
    steps = r.get("steps")
    if not isinstance(steps, int) or steps < 0:
        raise ConfigError('"run.steps" must be a non-negative integer')
    out = {"grid": {"shape": shape, "h": float(g.get("h", 1.0))},
           "model": {"name": m["name"], "coeffs": [float(c) for c in m["coeffs"]],
                     "dt": float(m["dt"]), "stencil": m.get("stencil", "std")},
           "init": dict(i),
           "run": {"steps": steps, "tuning": r.get("tuning", "auto"),
                   "series_every": int(r.get("series_every", max(1, steps))),
                   "energy": bool(r.get("energy", False)),
                   "series_path": r.get("series_path"),
                   "checkpoint_every": int(r.get("checkpoint_every", 0)),
                   "checkpoint_path": r.get("checkpoint_path", "ckpt_{step}.npz")}}
    t = out["run"]["tuning"]
    if not (t is None or t == "auto" or (isinstance(t, list) and len(t) == 3)):
        raise ConfigError('"run.tuning" must be "auto", null or [tile_x, tile_y, k]')
    if out["run"]["series_every"] < 1 or out["run"]["checkpoint_every"] < 0:
        raise ConfigError('"run.series_every" must be >= 1 and "run.checkpoint_every" >= 0')
    return out


def initial_fields(cfg: dict, shape):
    """The initial fields of a validated configuration (not for "checkpoint")."""
    i = cfg["init"]
    if "npy" in i:
        fields = [np.load(p) for p in i["npy"]]
    else:
        import synthetic  # the repository's seeded input recipes
        fn = getattr(synthetic, i["synthetic"], None)
        if fn is None or not callable(fn):
            raise ConfigError(f'no recipe "{i["synthetic"]}" in synthetic')
        out = fn(tuple(shape), **i.get("args", {}))
        fields = list(out) if isinstance(out, tuple) else [out]
    for f in fields:
        if tuple(f.shape) != tuple(shape):
            raise ConfigError(f"initial field of shape {f.shape}, expected {tuple(shape)}")
    return [np.ascontiguousarray(f, dtype=np.float32) for f in fields]


def run(cfg: dict) -> dict:
    """Execute a configuration; returns the summary (also what the command line prints)."""
    import paper_2109_02598_gb300 as pf
    cfg = validate(cfg)
    m, r = cfg["model"], cfg["run"]
    if "checkpoint" in cfg["init"]:
        g = pf.Grid.load(cfg["init"]["checkpoint"])
        if list(g.shape) != cfg["grid"]["shape"] or g.model != m["name"]:
            raise ConfigError("the checkpoint's grid or model differs from the configuration")
    else:
        g = pf.Grid(cfg["grid"]["shape"], MODELS[m["name"]], cfg["grid"]["h"])
        g.set_model(m["name"], m["coeffs"], m["dt"])
        if m["stencil"] != "std":
            g.set_stencil(m["stencil"])
        g.write_fields(initial_fields(cfg, cfg["grid"]["shape"]))
    if r["tuning"] == "auto":
        g.autotune()
    elif isinstance(r["tuning"], list):
        g.set_tuning(*r["tuning"])
    energy = r["energy"] and m["name"] != "gs"

    def sample():
        rec = {"step": g.steps_done, "mass": [g.mass(f) for f in range(g.n_fields)]}
        if energy:
            rec["energy"] = g.energy()
        return rec

    series, checkpoints = [sample()], []
    start, steps = g.steps_done, r["steps"]
    se, ce = r["series_every"], r["checkpoint_every"]
    done = 0
    while done < steps:
        # step to the next event: a series sample, a checkpoint or the end
        target = min((done // se + 1) * se, steps)
        if ce:
            target = min(target, (done // ce + 1) * ce)
        g.step(target - done)
        done = target
        if done % se == 0 or done == steps:
            series.append(sample())
        if ce and done % ce == 0:
            path = r["checkpoint_path"].format(step=g.steps_done)
            g.save(path)
            checkpoints.append(path)
    assert g.steps_done == start + steps
    if r["series_path"]:
        d = os.path.dirname(os.path.abspath(r["series_path"]))
        os.makedirs(d, exist_ok=True)
        with open(r["series_path"], "w") as f:
            json.dump(series, f, indent=1)
    summary = {"model": m["name"], "shape": cfg["grid"]["shape"], "steps": r["steps"],
               "steps_done": g.steps_done, "tuning": list(g.tuning), "series": len(series),
               "checkpoints": checkpoints, "final_mass": series[-1]["mass"]}
    g.close()
    return summary


def main(argv=None) -> int:
    argv = sys.argv[1:] if argv is None else argv
    if len(argv) != 1:
        print("usage: python -m paper_2109_02598_gb300.run config.json", file=sys.stderr)
        return 2
    with open(argv[0]) as f:
        cfg = json.load(f)
    try:
        print(json.dumps(run(cfg)))
    except ConfigError as e:
        print(f"configuration error: {e}", file=sys.stderr)
        return 2
    return 0


if __name__ == "__main__":
    sys.exit(main())
