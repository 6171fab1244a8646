"""Build the library's CUDA sources as host code for the CPU emulator.

The sources in paper_1703_04219_gb300/csrc are rewritten mechanically
(kernel launches ``k<<<g, b, smem, s>>>(args)`` become calls of
``emu_run_grid``; ``extern __shared__`` arrays become the per-block buffer)
and compiled with g++ and AddressSanitizer against ``fake/cuda_runtime.h``,
which runs every CUDA thread of a block as a host thread with barriers for
``__syncthreads``, ``__syncwarp`` and the warp shuffles.  Device buffers are
plain heap blocks of their exact size, so any out-of-bounds access of a
kernel is reported by the sanitizer.  Test infrastructure only.
"""
from __future__ import annotations

import os
import re
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
CSRC = os.path.join(ROOT, "paper_1703_04219_gb300", "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libp2emu.so")

_LAUNCH = re.compile(r'([A-Za-z_]\w*(?:<[^<>;()]*>)?)<<<')
_DYN = re.compile(r'extern __shared__ (?:__align__\(\d+\) )?([\w ]+?) (\w+)\[\];')


def convert(src: str) -> str:
    src = _DYN.sub(lambda m: f'{m.group(1)} *{m.group(2)} = '
                   f'reinterpret_cast<{m.group(1)} *>(emu_dyn_smem_ptr);', src)
    out, i = [], 0
    while True:
        m = _LAUNCH.search(src, i)
        if not m:
            out.append(src[i:])
            break
        out.append(src[i:m.start()])
        j = src.index('>>>', m.end())
        cfg = src[m.end():j]
        k = j + 3
        if src[k] != '(':
            raise ValueError(f"unexpected launch syntax near: {src[k - 40:k + 40]!r}")
        depth, p = 0, k
        while True:
            if src[p] == '(':
                depth += 1
            elif src[p] == ')':
                depth -= 1
                if depth == 0:
                    break
            p += 1
        out.append(f'emu_run_grid(emu_cfg({cfg}), [&]() {{ {m.group(1)}({src[k + 1:p]}); }})')
        i = p + 1
    return ''.join(out)


def _compile(args):
    r = subprocess.run(args, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"{' '.join(args)}\n{r.stderr[-4000:]}")


def build() -> str:
    gen = os.path.join(BUILD, "gen")
    os.makedirs(gen, exist_ok=True)
    units = []
    for f in sorted(os.listdir(CSRC)):
        if f.endswith((".cu", ".cuh")):
            with open(os.path.join(CSRC, f)) as fh:
                text = convert(fh.read())
            name = f[:-3] + ".cpp" if f.endswith(".cu") else f
            with open(os.path.join(gen, name), "w") as fh:
                fh.write(text)
            if f.endswith(".cu"):
                units.append(os.path.join(gen, name))
    units.append(os.path.join(HERE, "emu_rt.cpp"))
    flags = ["g++", "-std=c++20", "-O1", "-g", "-ffp-contract=off", "-fsanitize=address",
             "-fno-omit-frame-pointer", "-DP2_CPU_EMU",
             "-fPIC", "-I", os.path.join(HERE, "fake"), "-I", CSRC]
    objs = [os.path.join(BUILD, os.path.basename(u)[:-4] + ".o") for u in units]
    with ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        list(ex.map(_compile, [flags + ["-c", u, "-o", o] for u, o in zip(units, objs)]))
    _compile(["g++", "-shared", "-fsanitize=address", "-o", LIB] + objs)
    return LIB


if __name__ == "__main__":
    print(build())
    sys.exit(0)
