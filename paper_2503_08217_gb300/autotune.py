"""Autotuner for libs3r's launch shapes.

The tile is fixed at 16x16 pixels (the unit of work of the tiled alpha blend,
Eq. 2, as 3DGS rasterises); what is tuned is how the kernels map onto an SM:
the Gaussians staged in shared memory per batch of the blend forward and
backward, the resident blocks per SM that bound their register budgets, the
keys per thread of the onesweep radix tile, the outputs per thread of the
pair expansion, and the resident blocks of the projection pass. Every one is
a build-time define (``S3R_*``) with its default in the CUDA source; the
default values are this tuner's choice at the surround-rig workload.

Search: coordinate descent from the source defaults. For each parameter in
turn, every candidate value is built as a variant library
(``build.build(defines=...)``, which recompiles only the translation units
that see the define) and timed by running ``bench.py`` in a child process
with ``S3R_LIBRARY`` pointing at the variant; the step time (CUDA events,
after warm-up, on the full step: compaction, projection, LOD, sort, blend
forward and backward, visibility write-back) decides. A candidate replaces
the current value only when it is faster by more than ``--min-gain``.

    python -m paper_2503_08217_gb300.autotune --steps 10 --warmup 3 \\
        --out autotune.md [--params S3R_BLEND_FWD_BATCH,...] [--budget-s 600] [--write]

``--write`` rewrites the winning defaults into the sources. The timing runs
need a GPU; the search, the variant builds and ``--dry-run`` do not.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import os
import re
import subprocess
import sys
import time
from typing import Callable

from . import build as libbuild

ROOT = libbuild.ROOT


@dataclasses.dataclass(frozen=True)
class Param:
    name: str            # the build define
    source: str          # file under csrc/ holding its default
    candidates: tuple    # values tried (each legal under the source's static_asserts)
    what: str


PARAMS = (
    Param("S3R_BLEND_FWD_BATCH", "k_blend.cu", (32, 64, 128), "Gaussians staged per batch, blend forward"),
    Param("S3R_BLEND_FWD_BLOCKS", "k_blend.cu", (16, 20, 24), "resident blocks per SM, blend forward"),
    Param("S3R_BLEND_BWD_BATCH", "k_blend.cu", (32, 64, 128), "Gaussians staged per batch, blend backward"),
    Param("S3R_BLEND_BWD_BLOCKS", "k_blend.cu", (12, 16, 20), "resident blocks per SM, blend backward"),
    Param("S3R_SORT_ITEMS", "s3r_internal.cuh", (11, 15, 18), "keys per thread of a radix tile"),
    Param("S3R_SORT_BLOCKS", "s3r_internal.cuh", (2, 3, 4), "resident onesweep blocks per SM"),
    Param("S3R_SORT_LOOKBACK", "k_sort.cu", (4, 8, 16), "look-back words read per round trip, onesweep"),
    Param("S3R_DUP_EXPAND_ITEMS", "k_sort.cu", (4, 8, 12), "pairs written per thread, expansion"),
    Param("S3R_PROJECT_MASK_BLOCKS", "k_project.cu", (4, 6, 8), "resident blocks per SM, projection mask"),
)
BY_NAME = {p.name: p for p in PARAMS}

_DEFAULT_RE = r"^#ifndef {name}\n#define {name} (\d+)\b"


def source_defaults(csrc: str = libbuild.CSRC) -> dict:
    """The default of every tuned define, read from its ``#ifndef``/``#define``
    pair in the source."""
    out = {}
    for p in PARAMS:
        with open(os.path.join(csrc, p.source)) as f:
            m = re.search(_DEFAULT_RE.format(name=p.name), f.read(), re.M)
        if m is None:
            raise RuntimeError(f"{p.name}: no default in {p.source}")
        out[p.name] = int(m.group(1))
    return out


def write_defaults(values: dict, csrc: str = libbuild.CSRC) -> list:
    """Rewrite the defaults of ``values`` in the sources; returns the changed names."""
    changed = []
    for name, v in values.items():
        p = BY_NAME[name]
        path = os.path.join(csrc, p.source)
        with open(path) as f:
            text = f.read()
        pat = re.compile(_DEFAULT_RE.format(name=name), re.M)
        m = pat.search(text)
        if m is None:
            raise RuntimeError(f"{name}: no default in {p.source}")
        if int(m.group(1)) == v:
            continue
        text = text[:m.start(1)] + str(int(v)) + text[m.end(1):]
        with open(path, "w") as f:
            f.write(text)
        changed.append(name)
    return changed


def bench_record(lib: str | None, workload: str, steps: int, warmup: int,
                 timeout_s: float = 600.0) -> dict:
    """Time one library with ``bench.py`` in a child process; returns its JSON
    line (``ms_per_step``, and ``clocks``: the SM clock and throttle reasons
    sampled during the timed steps)."""
    env = dict(os.environ)
    if lib is None:
        env.pop("S3R_LIBRARY", None)
    else:
        env["S3R_LIBRARY"] = lib
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--workload", workload,
           "--steps", str(steps), "--warmup", str(warmup),
           "--no-plain", "--no-cpu", "--no-e2e", "--no-adam"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=timeout_s)
    if r.returncode != 0:
        raise RuntimeError(f"bench failed ({r.returncode}):\n{r.stderr[-2000:]}")
    for line in reversed(r.stdout.strip().splitlines()):
        if line.startswith("{"):
            return json.loads(line)
    raise RuntimeError("bench printed no JSON line")


def clock_note(rec: dict) -> str:
    """'<median SM MHz> / <max> MHz[, reasons]' from a bench line's clocks."""
    c = rec.get("clocks") or {}
    if not c.get("sm_mhz"):
        return "not sampled"
    reasons = ", ".join(c.get("reasons") or []) or "no reason"
    return f"{c['sm_mhz']:.0f} / {c.get('sm_max_mhz') or 0:.0f} MHz, {reasons}"


def coordinate_descent(start: dict, params, measure: Callable[[dict], float],
                       min_gain: float = 0.01, passes: int = 1,
                       deadline: float | None = None, log=None):
    """Minimise ``measure`` over one parameter at a time.

    ``start`` holds every parameter's current value; ``params`` lists the
    (name, candidates) pairs searched, in order. Returns (best values, best
    time, trials) with trials = [(values, time or error string)]. A candidate
    is accepted only when faster than the incumbent by more than ``min_gain``
    (relative). A configuration already timed is not timed again. Stops
    starting new trials once ``deadline`` (time.time()) passes.
    """
    cur = dict(start)
    trials = []
    seen = {}   # configuration -> time: each one is timed once

    def run(values):
        key = tuple(sorted(values.items()))
        if key in seen:
            return seen[key]
        try:
            t = measure(values)
        except Exception as e:   # a variant that fails to build or run is skipped
            t = f"{type(e).__name__}: {str(e).splitlines()[0] if str(e) else ''}"
        trials.append((dict(values), t))
        seen[key] = t
        if log:
            log(values, t)
        return t

    best = run(cur)
    if isinstance(best, str):
        raise RuntimeError(f"the starting configuration failed: {best}")
    for _ in range(passes):
        improved = False
        for name, cands in params:
            for v in cands:
                if v == cur[name]:
                    continue
                if deadline is not None and time.time() > deadline:
                    return cur, best, trials
                t = run({**cur, name: v})
                if not isinstance(t, str) and t < best * (1.0 - min_gain):
                    cur, best, improved = {**cur, name: v}, t, True
        if not improved:
            break
    return cur, best, trials


def report(start: dict, best: dict, best_ms: float, trials, workload: str, steps: int,
           warmup: int, notes: dict | None = None, retimed: float | None = None) -> str:
    """Markdown table of the trials; ``notes`` maps a configuration (sorted
    items) to a clock note, ``retimed`` is a second timing of the chosen one."""
    notes = notes or {}
    base = trials[0][1]
    lines = [f"# Launch-shape autotune, workload `{workload}` ({steps} timed steps after "
             f"{warmup} warm-up, one child process per trial)", "",
             "| trial | changed from start | ms / step | vs start | SM clock (median / max), reasons |",
             "|---|---|---|---|---|"]
    for i, (vals, t) in enumerate(trials):
        diff = ", ".join(f"{k}={v}" for k, v in vals.items() if v != start[k]) or "(start)"
        note = notes.get(tuple(sorted(vals.items())), "")
        if isinstance(t, str):
            lines.append(f"| {i} | {diff} | failed: {t} | | |")
        else:
            lines.append(f"| {i} | {diff} | {t:.3f} | {t / base:.3f} | {note} |")
    lines += ["", "| define | start | chosen |", "|---|---|---|"]
    for k in start:
        lines.append(f"| {k} | {start[k]} | {best[k]} |")
    lines += ["", f"best: {best_ms:.3f} ms / step (start {base:.3f})"]
    if retimed is not None:
        lines.append(f"chosen configuration timed again in a fresh process: {retimed:.3f} ms / step "
                     f"({100 * (retimed / best_ms - 1):+.2f} %: the run-to-run spread)")
    return "\n".join(lines) + "\n"


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--workload", default="rig")
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--params", default=None, help="comma-separated defines (default: all)")
    ap.add_argument("--candidates", action="append", default=[],
                    help="NAME=v1,v2,... overrides a parameter's candidate list")
    ap.add_argument("--min-gain", type=float, default=0.01)
    ap.add_argument("--passes", type=int, default=1)
    ap.add_argument("--budget-s", type=float, default=None,
                    help="start no new trial after this many seconds")
    ap.add_argument("--out", default=None, help="write the markdown report here")
    ap.add_argument("--write", action="store_true", help="write the winners into the sources")
    ap.add_argument("--dry-run", action="store_true", help="build every variant, time nothing")
    ap.add_argument("--no-retime", action="store_true",
                    help="skip the second timing of the chosen configuration")
    a = ap.parse_args(argv)

    start = source_defaults()
    names = [n.strip() for n in a.params.split(",")] if a.params else [p.name for p in PARAMS]
    cands = {n: BY_NAME[n].candidates for n in names}
    for spec in a.candidates:
        n, vs = spec.split("=", 1)
        if n not in BY_NAME:
            raise SystemExit(f"unknown define {n}")
        cands[n] = tuple(int(x) for x in vs.split(","))
        if n not in names:
            names.append(n)
    search = [(n, cands[n]) for n in names]

    def lib_for(values):
        diff = {k: v for k, v in values.items() if v != start[k]}
        return libbuild.build(defines=diff) if diff else libbuild.build()

    if a.dry_run:
        for n, cs in search:
            for v in cs:
                print(n, v, lib_for({**start, n: v}))
        return 0

    notes = {}

    def measure(values):
        rec = bench_record(lib_for(values), a.workload, a.steps, a.warmup)
        notes[tuple(sorted(values.items()))] = clock_note(rec)
        return float(rec["ms_per_step"])

    done = []   # (values, time) so far: the report is rewritten after every trial

    def log(values, t):
        diff = ", ".join(f"{k}={v}" for k, v in values.items() if v != start[k]) or "(start)"
        print(f"{diff}: {t if isinstance(t, str) else f'{t:.3f} ms'}", file=sys.stderr, flush=True)
        done.append((dict(values), t))
        if a.out and not isinstance(done[0][1], str):
            ok = [(v, x) for v, x in done if not isinstance(x, str)]
            bv, bt = min(ok, key=lambda vx: vx[1])
            with open(a.out, "w") as f:
                f.write(report(start, bv, bt, done, a.workload, a.steps, a.warmup, notes)
                        + "\n(partial: the search is still running)\n")

    deadline = time.time() + a.budget_s if a.budget_s else None
    best, best_ms, trials = coordinate_descent(start, search, measure, a.min_gain, a.passes,
                                               deadline, log)
    retimed = None
    if not a.no_retime:
        try:
            retimed = measure(best)
        except Exception as e:
            print(f"re-timing failed: {e}", file=sys.stderr)
    text = report(start, best, best_ms, trials, a.workload, a.steps, a.warmup, notes, retimed)
    print(text)
    if a.out:
        with open(a.out, "w") as f:
            f.write(text)
    if a.write:
        changed = write_defaults({k: v for k, v in best.items() if v != start[k]})
        print("rewrote:", ", ".join(changed) if changed else "nothing (the defaults won)")
    return 0


if __name__ == "__main__":
    sys.exit(main())
