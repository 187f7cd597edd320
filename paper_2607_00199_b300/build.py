"""Build libgb.so in-tree for sm_103a with nvcc (no GPU needed to build).

    python -m paper_2607_00199_b300.build [--verbose]

Object files go to _build/ at the repository root; the shared library is
written next to this file, where the ctypes binding loads it.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, 'csrc')
INCLUDE = os.path.join(ROOT, 'include')
BUILD = os.path.join(ROOT, '_build')
LIB = os.path.join(HERE, 'libgb.so')

SOURCES = ['gb_api.cpp', 'gb_reference.cpp', 'gb_kernels.cu', 'gb_kernels_tc.cu', 'gb_kernels_um.cu', 'gb_diagnostics.cu', 'gb_noalloc.cu',
           'gb3d.cpp', 'gb_kernels3d.cu', 'gb_kernels3d_tc.cu', 'gb_pml.cu']
ARCH = ['-gencode', 'arch=compute_103a,code=sm_103a']
FLAGS = ['-O3', '-lineinfo', '-std=c++17', '-Xcompiler', '-fPIC', '-I', INCLUDE, '-I', CSRC]


def _nvcc():
    cand = os.path.join(os.environ.get('CUDA_HOME', '/usr/local/cuda'), 'bin', 'nvcc')
    return cand if os.path.exists(cand) else 'nvcc'


def _compile(src, verbose):
    obj = os.path.join(BUILD, os.path.splitext(src)[0] + '.o')
    cmd = [_nvcc()] + ARCH + FLAGS + ['-c', os.path.join(CSRC, src), '-o', obj]
    if src.endswith('.cu'):
        cmd += ['-Xptxas', '-v'] if verbose else []
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError('nvcc failed for %s:\n%s\n%s' % (src, r.stdout, r.stderr))
    if verbose and (r.stdout or r.stderr):
        print(r.stdout + r.stderr)
    return obj


def build(verbose=False):
    os.makedirs(BUILD, exist_ok=True)
    with ThreadPoolExecutor(len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose), SOURCES))
    cmd = [_nvcc()] + ARCH + ['-shared', '-o', LIB] + objs + ['-lcudart']
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError('link failed:\n%s\n%s' % (r.stdout, r.stderr))
    return LIB


if __name__ == '__main__':
    print(build(verbose='--verbose' in sys.argv))
