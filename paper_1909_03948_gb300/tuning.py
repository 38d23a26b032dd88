"""Persistent table of autotuned solver settings.

Keys are (dim, N, nrhs, precision); values are the settings hp_autotune chose and
the milliseconds per block it measured.  The table is a JSON file (default
``$HP_TUNING_FILE`` or ``~/.cache/hp_gb300/tuning.json``).
"""
from __future__ import annotations

import json
import os

DEFAULT_PATH = os.environ.get("HP_TUNING_FILE", os.path.join(os.path.expanduser("~"), ".cache", "hp_gb300",
                                                                "tuning.json"))


def _key(problem, nrhs, precision):
    return f"d{problem.dim}_N{problem.N}_s{nrhs}_{precision}"


def load(path: str = DEFAULT_PATH) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save(table: dict, path: str = DEFAULT_PATH) -> None:
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tuned(problem, nrhs: int, precision: str = "fp32_ir", path: str = DEFAULT_PATH, retune: bool = False, X=None):
    """Applies the stored settings for this problem size and block width, running the
    autotuner (at the problem's current point, on the block X when given, else on a random
    block) when there are none.  Returns (settings, ms per block, 'table' | 'autotune')."""
    table = load(path)
    key = _key(problem, nrhs, precision)
    if key in table and not retune:
        s = table[key]["settings"]
        problem.set_tuning(**s)
        return s, table[key]["ms"], "table"
    s, ms = problem.autotune(nrhs, X=X)
    table[key] = {"settings": s, "ms": ms}
    save(table, path)
    return s, ms, "autotune"
