"""Build liblbm.so (the CUDA library behind include/lbm.h) in-tree for sm_103a.

The fifteen (stencil, storage) kernel units and the remaining units compile
in parallel with nvcc; a unit is recompiled only when a file its nvcc
dependency list names (or its command line) changed.  The shared library is
linked next to this file.
Run as ``python -m paper_2211_02435_b300.build [--force] [-v]``.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OBJ = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "liblbm.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         f"-I{INCLUDE}", f"-I{CSRC}"] + ARCH


def _deps():
    return (glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cuh"))
            + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(INCLUDE, "*.h"))
            + [os.path.abspath(__file__)])


def _units():
    units = []
    for st in range(3):
        for so in range(5):
            units.append((os.path.join(CSRC, "lbm_inst.cu"), f"inst_{st}_{so}.o",
                          [f"-DLBM_ST={st}", f"-DLBM_STORE={so}"]))
    for src in sorted(glob.glob(os.path.join(CSRC, "*.cu"))):
        if os.path.basename(src) != "lbm_inst.cu":
            units.append((src, os.path.basename(src)[:-3] + ".o", []))
    return units


STAMP = LIB + ".sha1"


def _sources_hash() -> str:
    import hashlib
    h = hashlib.sha1()
    for d in sorted(_deps()):
        h.update(os.path.relpath(d, ROOT).encode())
        with open(d, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def up_to_date() -> bool:
    """The library exists and was linked from the sources as they are now
    (content hash recorded next to it at link time)."""
    if not (os.path.exists(LIB) and os.path.exists(STAMP)):
        return False
    with open(STAMP) as fh:
        return fh.read().strip() == _sources_hash()


def _flags_of(extra):
    return " ".join([NVCC] + FLAGS + extra)


def _dep_files(out):
    """Repository files named by the nvcc dependency list of an object."""
    dep = out + ".d"
    if not os.path.exists(dep):
        return None
    text = open(dep).read().replace("\\\n", " ")
    files = text.split(":", 1)[1].split() if ":" in text else []
    return sorted({os.path.abspath(f) for f in files
                   if os.path.abspath(f).startswith(ROOT + os.sep)})


def _unit_stamp(src, out, extra, contents):
    """Hash of an object's command line and of the contents its repository
    dependencies had when this build started (`contents`: path -> bytes)."""
    import hashlib
    files = _dep_files(out)
    if files is None:
        return None
    h = hashlib.sha1(_flags_of(extra).encode())
    for f in sorted(set(files) | {os.path.abspath(src)}):
        if f not in contents:
            return None
        h.update(f.encode())
        h.update(contents[f])
    return h.hexdigest()


def _obj_current(src, out, extra, contents):
    """An object is current when its stamp matches its command line and the
    contents of the files it depends on; a file edited while it compiled
    leaves the stamp of the old contents, so the next build redoes it."""
    stamp = out + ".stamp"
    if not (os.path.exists(out) and os.path.exists(stamp)):
        return False
    want = _unit_stamp(src, out, extra, contents)
    return want is not None and open(stamp).read().strip() == want


def build(force: bool = False, jobs: int | None = None, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    stamp = _sources_hash()  # of the sources this build starts from
    contents = {}
    for d in _deps():
        with open(d, "rb") as fh:
            contents[os.path.abspath(d)] = fh.read()
    os.makedirs(OBJ, exist_ok=True)

    def compile_one(u):
        src, obj, extra = u
        out = os.path.join(OBJ, obj)
        if not force and _obj_current(src, out, extra, contents):
            return out
        cmd = [NVCC] + FLAGS + extra + ["-MD", "-MF", out + ".d", "-c", src, "-o", out]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {obj}:\n{r.stderr}")
        st = _unit_stamp(src, out, extra, contents)
        with open(out + ".stamp", "w") as fh:
            fh.write((st or "") + "\n")
        return out

    with cf.ThreadPoolExecutor(max_workers=jobs or os.cpu_count() or 4) as ex:
        objs = list(ex.map(compile_one, _units()))
    tmp = LIB + f".tmp{os.getpid()}"
    r = subprocess.run([NVCC] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"],
                       capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    with open(STAMP, "w") as fh:
        fh.write(stamp + "\n")
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
