"""Build libchase.so in-tree with nvcc for sm_103a (GB300).

Every translation unit under ``csrc/`` is compiled in parallel into
``_build/`` and linked into ``paper_1805_10121_gb300/libchase.so``.  An
object is rebuilt when the SHA-256 of its source, the headers, this script
and the compiler flags differs from the one recorded beside it (content, not
modification times, so a copied tree with stale objects still rebuilds).
``last_build`` records what the most recent ``build()`` of this process did.
"""

from __future__ import annotations

import concurrent.futures as cf
import glob
import hashlib
import json
import os
import platform
import shutil
import subprocess
import sys
import time

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libchase.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found")
    return cand


def _flags():
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
                   "-I", os.path.join(ROOT, "include"), "-I", CSRC]


def _digest(paths: list[str], extra: str) -> str:
    h = hashlib.sha256(extra.encode())
    for p in paths:
        h.update(os.path.basename(p).encode())
        with open(p, "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def _stale(out: str, digest: str) -> bool:
    """True unless ``out`` exists and was made from inputs with this digest."""
    try:
        with open(out + ".sha256") as f:
            return not os.path.exists(out) or f.read().strip() != digest
    except OSError:
        return True


def _record(out: str, digest: str) -> None:
    with open(out + ".sha256", "w") as f:
        f.write(digest + "\n")


def _record_library(digest: str) -> None:
    """Provenance of the linked library: source digest, machine, time."""
    with open(LIB + ".built", "w") as f:
        json.dump({"sources_sha256": digest, "machine": platform.machine(),
                   "built_at": time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime())}, f)


def library_provenance() -> dict:
    """Where and from which sources the current libchase.so was built, and
    whether it matches the sources in the tree now."""
    try:
        with open(LIB + ".built") as f:
            rec = json.load(f)
    except (OSError, ValueError):
        rec = {}
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))
    headers = sorted(glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.hpp"))
                     + glob.glob(os.path.join(ROOT, "include", "*.h"))) + [os.path.abspath(__file__)]
    flags = " ".join(_flags())
    objs = "".join(_digest([s] + headers, flags) for s in srcs)
    now = hashlib.sha256(objs.encode()).hexdigest()
    rec["matches_tree"] = rec.get("sources_sha256") == now and os.path.exists(LIB)
    return rec


# What the last build() of this process did: the translation units nvcc
# compiled, whether the library was linked, and the digest of all inputs.
last_build: dict = {"compiled": [], "linked": False, "sources_sha256": None}


def build(verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))
    headers = sorted(glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.hpp"))
                     + glob.glob(os.path.join(ROOT, "include", "*.h"))) + [os.path.abspath(__file__)]
    nv = nvcc()
    flags = " ".join(_flags())
    jobs = []
    objs = []
    digests = {}
    for s in srcs:
        o = os.path.join(BUILD, os.path.basename(s) + ".o")
        objs.append(o)
        dg = _digest([s] + headers, flags)
        digests[o] = dg
        if _stale(o, dg):
            lang = ["-x", "cu"] if s.endswith(".cu") else ["-x", "c++"]
            jobs.append((o, [nv] + _flags() + lang + ["-c", s, "-o", o]))

    def run(job):
        o, cmd = job
        r = subprocess.run(cmd, capture_output=True, text=True)
        return o, cmd, r

    compiled = []
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        for o, cmd, r in ex.map(run, jobs):
            if verbose or r.returncode != 0:
                sys.stderr.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed for {cmd[-3]}")
            _record(o, digests[o])
            compiled.append(os.path.basename(o)[:-2])
    lib_digest = hashlib.sha256("".join(digests[o] for o in objs).encode()).hexdigest()
    linked = False
    if compiled or _stale(LIB, lib_digest):
        cmd = [nv] + ARCH + ["-shared", "-o", LIB] + objs + ["-lcusolver", "-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            sys.stderr.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
            raise RuntimeError("link of libchase.so failed")
        _record(LIB, lib_digest)
        _record_library(lib_digest)
        linked = True
    last_build.update(compiled=compiled, linked=linked, sources_sha256=lib_digest)
    if compiled or linked:
        sys.stderr.write(f"libchase: nvcc compiled {len(compiled)} translation unit(s), "
                         f"linked {os.path.basename(LIB)}\n")
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
