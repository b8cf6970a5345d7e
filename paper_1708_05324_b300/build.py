"""Build libgmmnlse.so (all CUDA sources under csrc/) for sm_103a, in-tree.

    python -m paper_1708_05324_b300.build [--force]
"""
import hashlib
import os
import subprocess
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libgmmnlse.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")

FLAGS = [
    "-gencode", "arch=compute_103a,code=sm_103a",
    "-O3", "-lineinfo", "-std=c++17",
    "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
    "--expt-relaxed-constexpr",
    "-I", os.path.join(ROOT, "include"),
]


def sources():
    out = []
    for name in sorted(os.listdir(CSRC)):
        if name.endswith((".cu", ".cuh", ".h")):
            out.append(os.path.join(CSRC, name))
    out.append(os.path.join(ROOT, "include", "gmmnlse.h"))
    return out


def _includes(path, seen=None):
    """The file and every local header it includes, transitively."""
    import re
    seen = set() if seen is None else seen
    if path in seen or not os.path.exists(path):
        return seen
    seen.add(path)
    with open(path) as f:
        for inc in re.findall(r'^\s*#\s*include\s+"([^"]+)"', f.read(), re.M):
            _includes(os.path.normpath(os.path.join(os.path.dirname(path), inc)), seen)
    return seen


def _unit_stamp(src):
    h = hashlib.sha256()
    h.update(" ".join(FLAGS).encode())
    for p in sorted(_includes(src)):
        h.update(p.encode())
        with open(p, "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def _stamp():
    h = hashlib.sha256()
    for p in sources():
        h.update(p.encode())
        with open(p, "rb") as f:
            h.update(f.read())
    h.update(" ".join(FLAGS).encode())
    return h.hexdigest()


def build(force=False, verbose=False, jobs=None):
    """Compile every translation unit under csrc/ whose sources changed (its
    own hash of the unit and the headers it includes) and link the library."""
    stamp_file = LIB + ".stamp"
    stamp = _stamp()
    if not force and os.path.exists(LIB) and os.path.exists(stamp_file):
        if open(stamp_file).read().strip() == stamp:
            return LIB
    objs = []
    build_dir = os.path.join(HERE, "_build")
    os.makedirs(build_dir, exist_ok=True)
    cu = [p for p in sources() if p.endswith(".cu")]
    todo = []
    for src in cu:
        obj = os.path.join(build_dir, os.path.basename(src) + ".o")
        objs.append(obj)
        us = _unit_stamp(src)
        ok = (not force and os.path.exists(obj) and os.path.exists(obj + ".stamp")
              and open(obj + ".stamp").read().strip() == us)
        if not ok:
            cmd = [NVCC, *FLAGS, "-c", src, "-o", obj]
            if verbose:
                cmd.insert(1, "-Xptxas=-v")
            todo.append((cmd, obj, us))
    # the slowest units first (the long-step drivers and the widest GEMM
    # instantiations), at most `jobs` compilers at once
    slow = ("persist_", "prop_", "tc_lsum_", "tc_store", "noalloc")
    todo.sort(key=lambda t: next((i for i, k in enumerate(slow) if k in os.path.basename(t[1])), len(slow)))
    jobs = jobs or max(1, os.cpu_count() or 1)
    running, failed = [], None
    while (todo and failed is None) or running:
        while todo and failed is None and len(running) < jobs:
            cmd, obj, us = todo.pop(0)
            running.append((cmd, obj, us, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        time.sleep(0.2)
        for r in list(running):
            cmd, obj, us, pr = r
            if pr.poll() is None:
                continue
            running.remove(r)
            out = pr.stdout.read()
            if pr.returncode != 0:
                failed = failed or ("nvcc failed:\n" + " ".join(cmd) + "\n" + out.decode(errors="replace"))
                continue
            if verbose and out:
                sys.stdout.write(out.decode(errors="replace"))
            with open(obj + ".stamp", "w") as f:
                f.write(us)
    if failed:
        raise RuntimeError(failed)
    tmp = LIB + ".tmp"
    cmd = [NVCC, "-gencode", "arch=compute_103a,code=sm_103a", "-shared", "-o", tmp, *objs, "-lcuda", "-ldl"]
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + " ".join(cmd) + "\n" + r.stdout.decode(errors="replace"))
    os.replace(tmp, LIB)
    with open(stamp_file, "w") as f:
        f.write(stamp)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
