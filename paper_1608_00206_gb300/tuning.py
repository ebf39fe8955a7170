"""Autotuned schedules.

``autotune`` runs the library's autotuner (hc_autotune: every candidate
schedule timed with CUDA events) for one (D, dtype); ``tune_table`` does it
for a range of D and dtypes and ``save`` writes the result as JSON.  The
table shipped with the package (``tuned_schedules.json``, produced on a GB300
by ``python -m paper_1608_00206_gb300.tuning``) is installed as the
library's per-(D, dtype) default (hc_set_default_schedule) the first time a
convolution runs on a device of the same name; a schedule changes speed only,
never the result bits.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import threading

import torch

from . import _lib
from ._lib import check

TABLE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned_schedules.json")
_DT = {"int64": (torch.int64, _lib.HC_INT64), "float64": (torch.float64, _lib.HC_FP64),
       "float32": (torch.float32, _lib.HC_FP32), "mixed": (torch.float32, _lib.HC_FP32_MIXED),
       "ff": (torch.float32, _lib.HC_FP32_FF)}
_installed = set()
_lock = threading.Lock()


def autotune(D: int, dtype: str = "int64", reps: int = 3, device=None):
    """(schedule dict, best ms) for one (D, dtype) on the current device."""
    tdt, code = _DT[dtype]
    dev = device or torch.device("cuda", torch.cuda.current_device())
    g = torch.Generator(device="cpu").manual_seed(D)
    if tdt == torch.int64:
        x = torch.randint(-1000, 1001, (1 << D,), generator=g, dtype=torch.int64).to(dev)
        y = torch.randint(-1000, 1001, (1 << D,), generator=g, dtype=torch.int64).to(dev)
    else:
        x = torch.rand(1 << D, generator=g, dtype=tdt).to(dev)
        y = torch.rand(1 << D, generator=g, dtype=tdt).to(dev)
    z = torch.empty(3 ** D, dtype=tdt, device=dev)
    lib = _lib.lib()
    nb = int(lib.hc_autotune_workspace_size(D, code))
    ws = torch.empty(max(nb, 256), dtype=torch.uint8, device=dev)
    best = _lib.hc_schedule()
    ms = ctypes.c_double()
    st = torch.cuda.current_stream(dev).cuda_stream
    check(lib.hc_autotune(x.data_ptr(), y.data_ptr(), z.data_ptr(), D, code, ws.data_ptr(), nb,
                          reps, st, ctypes.byref(best), ctypes.byref(ms)), "hc_autotune")
    return best.as_dict(), float(ms.value)


def tune_table(dims, dtypes, reps: int = 3):
    table = {"device": torch.cuda.get_device_name(), "schedules": {}}
    for dt in dtypes:
        for D in dims:
            s, ms = autotune(D, dt, reps)
            s["ms"] = round(ms, 5)
            table["schedules"].setdefault(dt, {})[str(D)] = s
            print(json.dumps({"dtype": dt, "D": D, **s}), flush=True)
            torch.cuda.empty_cache()
    return table


def save(table, path: str = TABLE):
    with open(path, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
        f.write("\n")


def install(table) -> int:
    """Install every entry of `table` as the library default; returns the count."""
    lib = _lib.lib()
    n = 0
    for dt, entries in table.get("schedules", {}).items():
        code = _DT[dt][1]
        for D, s in entries.items():
            sched = _lib.hc_schedule(s["kind"], s["c"], s["k"], s["cols"], s.get("cols_outer", 0),
                                     s.get("top", 0))
            check(lib.hc_set_default_schedule(int(D), code, ctypes.byref(sched)),
                  "hc_set_default_schedule")
            n += 1
    return n


def ensure_installed(device) -> None:
    """Install the shipped table once per process if it was tuned on a device
    with this device's name."""
    name = torch.cuda.get_device_name(device)
    with _lock:
        if name in _installed:
            return
        _installed.add(name)
        if not os.path.exists(TABLE):
            return
        with open(TABLE) as f:
            table = json.load(f)
        if table.get("device") == name:
            install(table)


def main():
    ap = argparse.ArgumentParser(description="tune schedules on this GPU")
    ap.add_argument("--dims", default="10-20")
    ap.add_argument("--dtypes", default="int64,float64,float32,mixed,ff")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--out", default=TABLE)
    a = ap.parse_args()
    lo, hi = (int(v) for v in a.dims.split("-"))
    from .build import build
    build()
    table = tune_table(range(lo, hi + 1), a.dtypes.split(","), a.reps)
    save(table, a.out)


if __name__ == "__main__":
    main()
