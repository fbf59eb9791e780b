"""Build libs3r.so (sm_103a) in-tree with nvcc: one object per translation
unit, compiled in parallel, then one shared-library link. No torch headers
are involved: the library's ABI is plain C (include/s3r.h).

Variant builds. The launch shapes (staged batch sizes, resident blocks per SM,
keys or outputs per thread) are build-time defines with defaults in the CUDA
sources. ``build(defines={...})`` links a variant library under
``_build/variants/<tag>/`` that the autotuner times; a variant recompiles only
the translation units whose text (or the project headers they include)
mentions one of its defines and reuses the default build's other objects.
"""
from __future__ import annotations

import concurrent.futures
import hashlib
import os
import re
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libs3r.so")
ARCH = "103a"

SOURCES = ["s3r_api.cu", "k_compact.cu", "k_project.cu", "k_sort.cu", "k_blend.cu",
           "k_project_bwd.cu", "k_vis.cu", "k_probe.cu", "k_ode.cu", "k_world.cu"]

_DEFINE_NAME = re.compile(r"^S3R_[A-Z0-9_]+$")


def nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libs3r")
    return cand


def _flags(verbose_ptxas: bool):
    f = ["-gencode", f"arch=compute_{ARCH},code=sm_{ARCH}", "-lineinfo", "-O3", "-std=c++17",
         "-I" + INCLUDE, "-Xcompiler", "-fPIC", "-DS3R_ARCH=103"]
    if verbose_ptxas:
        f += ["-Xptxas", "-v"]
    return f


def _deps_mtime() -> float:
    paths = [os.path.join(CSRC, p) for p in os.listdir(CSRC)] + [os.path.join(INCLUDE, "s3r.h")]
    return max(os.path.getmtime(p) for p in paths)


def unit_text(src: str) -> str:
    """The text of a translation unit and of every project header it includes
    (quoted includes found in csrc/ or include/, followed recursively)."""
    seen, out, todo = set(), [], [os.path.join(CSRC, src)]
    while todo:
        path = todo.pop()
        if path in seen:
            continue
        seen.add(path)
        with open(path) as f:
            text = f.read()
        out.append(text)
        for name in re.findall(r'^\s*#\s*include\s+"([^"]+)"', text, re.M):
            for d in (os.path.dirname(path), CSRC, INCLUDE):
                cand = os.path.join(d, name)
                if os.path.exists(cand):
                    todo.append(cand)
                    break
    return "\n".join(out)


def relevant_defines(src: str, defines: dict) -> dict:
    """The subset of ``defines`` that the unit ``src`` can see."""
    text = unit_text(src)
    return {k: defines[k] for k in sorted(defines) if re.search(r"\b%s\b" % k, text)}


def _check_defines(defines: dict) -> dict:
    out = {}
    for k, v in defines.items():
        if not _DEFINE_NAME.match(k):
            raise ValueError(f"{k!r} is not an S3R_ build define")
        if not isinstance(v, int) or isinstance(v, bool):
            raise ValueError(f"{k} must be an integer, got {v!r}")
        out[k] = v
    return out


def variant_tag(defines: dict) -> str:
    """Directory name of a variant: the defines, lower-cased, in name order."""
    return "-".join(f"{k[4:].lower()}{defines[k]}" for k in sorted(defines))


def variant_path(defines: dict) -> str:
    return os.path.join(BUILD, "variants", variant_tag(defines), "libs3r.so")


def _compile(cc, flags, src, obj, defines, quiet, verbose_ptxas):
    cmd = [cc, *flags, *[f"-D{k}={v}" for k, v in sorted(defines.items())],
           "-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    if not quiet or verbose_ptxas:
        sys.stderr.write(r.stderr)
    return obj


def _link(cc, objs, lib):
    tmp = lib + ".tmp"
    cmd = [cc, "-shared", "-gencode", f"arch=compute_{ARCH},code=sm_{ARCH}", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


def build(force: bool = False, verbose_ptxas: bool = False, quiet: bool = True,
          defines: dict | None = None) -> str:
    """Build the default library (no ``defines``) or a variant; returns its path."""
    if defines:
        return _build_variant(_check_defines(defines), force, verbose_ptxas, quiet)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _deps_mtime():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    flags = _flags(verbose_ptxas)

    def compile_one(src):
        return _compile(cc, flags, src, os.path.join(BUILD, src.replace(".cu", ".o")), {},
                        quiet, verbose_ptxas)

    with concurrent.futures.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    return _link(cc, objs, LIB)


def _build_variant(defines: dict, force: bool, verbose_ptxas: bool, quiet: bool) -> str:
    build(verbose_ptxas=verbose_ptxas, quiet=quiet)   # the default objects it reuses
    lib = variant_path(defines)
    deps = max(_deps_mtime(), os.path.getmtime(LIB))
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= deps:
        return lib
    os.makedirs(os.path.dirname(lib), exist_ok=True)
    obj_dir = os.path.join(BUILD, "variant_objs")
    os.makedirs(obj_dir, exist_ok=True)
    cc = nvcc()
    flags = _flags(verbose_ptxas)
    jobs, objs = [], []
    for src in SOURCES:
        rel = relevant_defines(src, defines)
        if not rel:
            objs.append(os.path.join(BUILD, src.replace(".cu", ".o")))
            continue
        key = hashlib.sha256(repr(sorted(rel.items())).encode()).hexdigest()[:12]
        obj = os.path.join(obj_dir, src.replace(".cu", f"-{key}.o"))
        objs.append(obj)
        if force or not os.path.exists(obj) or os.path.getmtime(obj) < deps:
            jobs.append((src, obj, rel))
    if jobs:
        with concurrent.futures.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
            list(ex.map(lambda j: _compile(cc, flags, j[0], j[1], j[2], quiet, verbose_ptxas),
                        jobs))
    return _link(cc, objs, lib)


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv, quiet=False))
