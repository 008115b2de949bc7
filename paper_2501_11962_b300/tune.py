"""Autotuning of the neighbour-search geometry with a JSON cache keyed by system shape.

The tuned quantities (cluster-column width, pair-search bin width) change only how many pairs
the kernels evaluate and how long the list build takes, never a result.  mop_autotune times
full evaluations on the GPU; this module remembers the winner per shape so later handles of the
same shape reuse it without timing again.
"""
from __future__ import annotations

import json
import os
from pathlib import Path

DEFAULT_CACHE = Path(os.environ.get("MOP_TUNE_CACHE", Path.home() / ".cache" / "mop_autotune.json"))


def shape_key(engine, path_id: int) -> str:
    s = engine.system
    n = engine.n_beads[path_id]
    return (f"Q{s.n_atoms}_box{s.box[0]:.4f}x{s.box[1]:.4f}x{s.box[2]:.4f}_rc{s.rc:.3f}_N{n}"
            f"_nt{s.n_types}_prec{engine.precision}")


def autotune(engine, path_id: int = 0, cache: Path | str | None = DEFAULT_CACHE, force: bool = False) -> dict:
    """Apply the cached tuning for this shape, or measure one with mop_autotune and cache it."""
    key = shape_key(engine, path_id)
    data = {}
    if cache is not None and Path(cache).exists():
        try:
            data = json.loads(Path(cache).read_text())
        except (OSError, ValueError):
            data = {}
    if key in data and not force:
        t = data[key]
        engine.set_tuning(t["col_factor"], t["bin_factor"])
        return dict(t, cached=True)
    t, ms = engine.autotune(path_id)
    rec = dict(t, ms_per_eval=ms)
    if cache is not None:
        data[key] = rec
        Path(cache).parent.mkdir(parents=True, exist_ok=True)
        tmp = Path(str(cache) + ".tmp")
        tmp.write_text(json.dumps(data, indent=1, sort_keys=True))
        tmp.replace(cache)
    return dict(rec, cached=False)
