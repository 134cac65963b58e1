"""Tuning cache for the x-z kernel variant of a plan.

ef_plan_autotune times the variants a plan supports on one sample snapshot;
this module remembers the winner per (grids, filter width, precision, wall
treatment) in a JSON file so later runs apply it with ef_plan_set_variant
instead of timing again.
"""
from __future__ import annotations

import json
import os

from . import eles

DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "autotune.json")


def plan_key(plan) -> str:
    d, l = plan.dns, plan.les
    return (f"{d.nx}x{d.ny}x{d.nz}->{l.nx}x{l.ny}x{l.nz}|L={d.Lx:.6g},{d.Lz:.6g}|"
            f"delta={plan.delta:.9g}|prec={plan.precision}")


def tune(plan, u, ubar, tau, cache_path: str = DEFAULT_CACHE, reps: int = 3) -> dict:
    """Apply the cached choice for this plan, or time the variants and cache
    the fastest.  Returns {"choice", "ms" (None when cached), "cached"}."""
    cache = {}
    if os.path.exists(cache_path):
        try:
            cache = json.load(open(cache_path))
        except (OSError, ValueError):
            cache = {}
    key = plan_key(plan)
    if key in cache:
        try:
            eles.plan_set_variant(plan, cache[key]["choice"])
            return {"choice": cache[key]["choice"], "ms": cache[key].get("ms"), "cached": True}
        except eles.EFError:
            pass
    choice, ms = eles.plan_autotune(plan, u, ubar, tau, reps)
    cache[key] = {"choice": choice, "ms": ms}
    os.makedirs(os.path.dirname(cache_path), exist_ok=True)
    tmp = cache_path + f".{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, cache_path)
    return {"choice": choice, "ms": ms, "cached": False}
