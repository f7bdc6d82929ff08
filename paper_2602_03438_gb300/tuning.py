"""Tile-shape autotuning of the sliced block products, kept as a JSON file.

``tune`` runs ``negf_tune_products`` (the library times every tile variant that supports
a block size on synthetic products and keeps the fastest for its context) for each
block size, and writes the choices with their timings to ``path``; ``load`` sets saved
choices on a context with ``negf_set_product_variant``.  File format:

    {"gpu": "<device name>", "units": U,
     "choices": {"<n>": {"variant": v, "ms": {"1": t1, "2": t2, "3": t3}}}}

Variants: 1 half-width tiles, 2 persistent full-width tiles, 3 full-width tiles (one CTA
per tile), 0 the built-in rule.  Marshalling and file handling only: the timing and the
choice are made by the library.
"""
from __future__ import annotations

import ctypes as C
import json
from typing import Iterable, Optional

import torch

from . import negf

VARIANTS = {0: "built-in rule", 1: "half-width tiles", 2: "persistent full-width tiles", 3: "full-width tiles"}


def tune(ctx: "negf.Context", sizes: Iterable[int], units: int = 1024, path: Optional[str] = None,
         stream=None) -> dict:
    """Tunes every block size in `sizes` on `units` products each; returns (and writes to
    `path` when given) the choices."""
    out = {"gpu": torch.cuda.get_device_name(ctx.device), "units": int(units), "choices": {}}
    for n in sorted(set(int(x) for x in sizes)):
        choice = C.c_int32(0)
        ms = (C.c_double * 4)()
        ctx.check(ctx.lib.negf_tune_products(ctx.h, n, int(units), C.byref(choice), ms, negf._stream(stream)))
        out["choices"][str(n)] = {"variant": int(choice.value),
                                  "ms": {str(v): float(ms[v]) for v in (1, 2, 3) if ms[v] >= 0.0}}
    if path:
        with open(path, "w") as f:
            json.dump(out, f, indent=1)
    return out


def load(ctx: "negf.Context", path: str) -> dict:
    """Sets the choices saved by `tune` on the context; returns them."""
    with open(path) as f:
        saved = json.load(f)
    for n, ent in saved.get("choices", {}).items():
        ctx.check(ctx.lib.negf_set_product_variant(ctx.h, int(n), int(ent["variant"])))
    return saved
