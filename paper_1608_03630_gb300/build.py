"""Build libreg.so (the C-ABI CUDA library) in-tree for sm_103a.

Each translation unit under csrc/ is compiled by nvcc in parallel into
``_build/`` and linked, with cuFFT and the shared CUDA runtime, into
``libreg.so`` beside this file.  The build is skipped when the library is
newer than every source and header.
"""

import concurrent.futures as cf
import glob
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, 'csrc')
INCLUDE = os.path.join(ROOT, 'include')
BUILD = os.path.join(HERE, '_build')
LIB = os.path.join(HERE, 'libreg.so')
ARCH = ['-gencode', 'arch=compute_103a,code=sm_103a']


def nvcc():
    cand = os.path.join(os.environ.get('CUDA_HOME', '/usr/local/cuda'), 'bin', 'nvcc')
    return cand if os.path.exists(cand) else 'nvcc'


def cuda_lib_dir():
    home = os.environ.get('CUDA_HOME', '/usr/local/cuda')
    for d in ('lib64', 'lib', os.path.join('targets', 'sbsa-linux', 'lib'),
              os.path.join('targets', 'x86_64-linux', 'lib')):
        p = os.path.join(home, d)
        if os.path.exists(os.path.join(p, 'libcufft.so')):
            return p
    return os.path.join(home, 'lib64')


def sources():
    return sorted(glob.glob(os.path.join(CSRC, '*.cu')))


def _stale():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = sources() + glob.glob(os.path.join(CSRC, '*.h')) + \
        glob.glob(os.path.join(CSRC, '*.cuh')) + glob.glob(os.path.join(INCLUDE, '*.h'))
    return any(os.path.getmtime(p) > t for p in deps)


def _compile(src, extra):
    obj = os.path.join(BUILD, os.path.basename(src).replace('.cu', '.o'))
    cmd = [nvcc(), '-c', src, '-o', obj, '-O3', '-std=c++17', '-lineinfo', *ARCH,
           '-Xcompiler', '-fPIC', '-I', INCLUDE, '-I', CSRC, *extra]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError('nvcc failed for %s:\n%s\n%s' % (src, ' '.join(cmd), r.stderr))
    return obj, r.stderr


def build(force=False, verbose=False, extra=()):
    """Compile and link libreg.so; returns its path."""
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        results = list(ex.map(lambda s: _compile(s, list(extra)), sources()))
    objs = [o for o, _ in results]
    if verbose:
        for _, err in results:
            if err.strip():
                print(err)
    libdir = cuda_lib_dir()
    tmp = LIB + '.tmp'
    cmd = [nvcc(), '-shared', '-o', tmp, *objs, *ARCH, '-cudart', 'shared',
           '-L', libdir, '-lcufft', '-Xlinker', '-rpath,' + libdir]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError('link failed:\n%s\n%s' % (' '.join(cmd), r.stderr))
    os.replace(tmp, LIB)
    return LIB


if __name__ == '__main__':
    import sys
    print(build(force='--force' in sys.argv, verbose=True,
                extra=['-Xptxas', '-v'] if '--ptxas' in sys.argv else []))
