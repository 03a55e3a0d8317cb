"""Build libvp.so in-tree with nvcc for sm_103a (one -gencode, translation units in parallel).

The library is rebuilt whenever the digest of its sources differs from the one it was
built from: a SHA-256 over every file under csrc/ and include/, this script and the
compile flags.  The digest is compiled into the library (vp_version() ends with it) and
recorded beside the build objects, so a library copied in from elsewhere or built from
other sources is never reused.
"""
from __future__ import annotations

import concurrent.futures
import hashlib
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libvp.so")

SOURCES = ["vp_api.cu", "vp_sweeps.cu", "vp_kernels.cu", "vp_static.cu", "vp_sweeps2_part0.cu",
           "vp_sweeps2_part1.cu", "vp_sweeps2_part2.cu", "fno.cu", "vp_vec.cu", "vp_vie.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libvp.so")
    return exe


def _flags(verbose: bool, debug: bool = False) -> list:
    f = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-fvisibility=hidden",
         "-I", INCLUDE, "-I", CSRC, *ARCH]
    if verbose:
        f += ["-Xptxas", "-v"]
    if debug:
        f += ["-DVP_DEBUG_CHECKS"]
    return f


def source_digest(debug: bool = False) -> str:
    """SHA-256 (first 16 hex digits) of the library's sources, this script and the flags."""
    h = hashlib.sha256()
    files = [os.path.join(CSRC, f) for f in sorted(os.listdir(CSRC))] + \
            [os.path.join(INCLUDE, f) for f in sorted(os.listdir(INCLUDE))] + [os.path.abspath(__file__)]
    for path in files:
        if not os.path.isfile(path):
            continue
        h.update(os.path.basename(path).encode() + b"\0")
        with open(path, "rb") as fh:
            h.update(fh.read())
        h.update(b"\0")
    h.update(" ".join(_flags(False, debug)).replace(ROOT, "").encode())
    return h.hexdigest()[:16]


DIGEST_FILE = os.path.join(BUILD, "libvp.digest")


def _compile(src: str, verbose: bool, debug: bool, digest: str) -> tuple:
    obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
    cmd = [nvcc(), "-c", os.path.join(CSRC, src), "-o", obj, *_flags(verbose, debug),
           f"-DVP_SOURCE_DIGEST=\"{digest}\""]
    r = subprocess.run(cmd, capture_output=True, text=True)
    return src, obj, r.returncode, r.stdout + r.stderr


def _stale(digest: str) -> bool:
    """True unless libvp.so exists and was built from sources with this digest."""
    if not os.path.exists(LIB) or not os.path.exists(DIGEST_FILE):
        return True
    with open(DIGEST_FILE) as fh:
        return fh.read().strip() != digest


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    """Compile every CUDA source and link libvp.so next to this file; return its path.

    debug=True adds the kernels' bounds self-checks (VP_DEBUG_CHECKS)."""
    digest = source_digest(debug)
    if not force and not _stale(digest):
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    if os.path.exists(DIGEST_FILE):
        os.remove(DIGEST_FILE)
    with concurrent.futures.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(lambda s: _compile(s, verbose, debug, digest), SOURCES))
    failed = [r for r in results if r[2] != 0]
    for src, _, rc, out in results:
        if verbose or rc != 0:
            sys.stderr.write(f"--- {src} (rc={rc})\n{out}\n")
    if failed:
        raise RuntimeError("nvcc failed for " + ", ".join(r[0] for r in failed))
    tmp = LIB + ".tmp"
    cmd = [nvcc(), "-shared", "-o", tmp, *[r[1] for r in results], *ARCH, "-lcudart_static"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link of libvp.so failed:\n" + r.stdout + r.stderr)
    os.replace(tmp, LIB)
    with open(DIGEST_FILE, "w") as fh:
        fh.write(digest + "\n")
    sys.stderr.write(f"libvp.so built from sources {digest}\n")
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv, debug="--debug" in sys.argv)
    print(LIB)
