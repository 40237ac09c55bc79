"""Compile the CUDA library (csrc/*.cu) for sm_103a into _lib/libokmc.so.

Plain nvcc, one object per translation unit compiled in parallel, then one link.
"""
from __future__ import annotations

import hashlib
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(HERE, 'csrc')
OUT = os.path.join(HERE, '_lib')
LIB = os.path.join(OUT, 'libokmc.so')
SOURCES = ['solve.cu', 'solve_fast.cu', 'defects.cu', 'dipole.cu', 'dislocation.cu', 'shift.cu', 'okmc_api.cu', 'serve.cu']
ARCH = ['-gencode', 'arch=compute_103a,code=sm_103a']
FLAGS = ['-O3', '-lineinfo', '-std=c++17', '-Xcompiler', '-fPIC', '-I' + os.path.join(ROOT, 'include')]


def nvcc_path():
    for cand in (os.environ.get('NVCC'), shutil.which('nvcc'), '/usr/local/cuda/bin/nvcc'):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError('nvcc not found')


STAMP = LIB + '.sha256'


def source_hash():
    """SHA-256 over the sources, the public header, this script and the compiler flags."""
    h = hashlib.sha256()
    deps = sorted(os.path.join(SRC, f) for f in os.listdir(SRC)) + [os.path.join(ROOT, 'include', 'okmc.h'), __file__]
    for p in deps:
        h.update(os.path.basename(p).encode())
        with open(p, 'rb') as f:
            h.update(f.read())
    h.update(' '.join(ARCH + FLAGS).encode())
    return h.hexdigest()


def _stale(digest):
    # keyed on content, not on modification times: a library copied next to its sources
    # with newer times is still rebuilt unless it was built from exactly these sources
    if not os.path.exists(LIB) or not os.path.exists(STAMP):
        return True
    with open(STAMP) as f:
        return f.read().strip() != digest


def build(force=False, verbose=False):
    """Build the library unless it was built from the current sources; return its path."""
    digest = source_hash()
    if not force and not _stale(digest):
        return LIB
    os.makedirs(OUT, exist_ok=True)
    nvcc = nvcc_path()
    procs = []
    objs = []
    for s in SOURCES:
        obj = os.path.join(OUT, s.replace('.cu', '.o'))
        objs.append(obj)
        cmd = [nvcc] + ARCH + FLAGS + ['-c', os.path.join(SRC, s), '-o', obj]
        if verbose:
            print(' '.join(cmd), file=sys.stderr)
        procs.append((s, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    errs = []
    for s, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            errs.append('%s:\n%s' % (s, out.decode(errors='replace')))
    if errs:
        raise RuntimeError('nvcc failed:\n' + '\n'.join(errs))
    tmp = LIB + '.tmp'
    cmd = [nvcc] + ARCH + ['-shared', '-o', tmp] + objs
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        raise RuntimeError('link failed:\n' + r.stdout.decode(errors='replace'))
    os.replace(tmp, LIB)
    with open(STAMP, 'w') as f:
        f.write(digest + '\n')
    return LIB


if __name__ == '__main__':
    print(build(force='--force' in sys.argv, verbose=True))
