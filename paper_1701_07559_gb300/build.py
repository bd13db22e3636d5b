"""Compile libmdwf.so in-tree for sm_103a (nvcc, one -gencode, sources in parallel)."""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, 'csrc')
BUILD = os.path.join(HERE, '_build')
LIB = os.path.join(HERE, 'libmdwf.so')
SOURCES = ['hop.cu', 'hop_fast.cu', 'hop_pair.cu', 'blas.cu', 'flow.cu', 'lib.cu']
NVCC_FLAGS = ['-gencode', 'arch=compute_103a,code=sm_103a', '-O3', '-lineinfo', '-std=c++17',
              '-Xcompiler', '-fPIC', '-Xcompiler', '-ffp-contract=off']


def _nvcc():
    cand = os.path.join(os.environ.get('CUDA_HOME', '/usr/local/cuda'), 'bin', 'nvcc')
    return cand if os.path.exists(cand) else 'nvcc'


def _deps():
    hdrs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith('.h')]
    hdrs.append(os.path.join(os.path.dirname(HERE), 'include', 'mdwf.h'))
    return hdrs


def build(force=False, verbose=False):
    """Build libmdwf.so if any source or header is newer than it.  Returns its path."""
    os.makedirs(BUILD, exist_ok=True)
    newest = max(os.path.getmtime(p) for p in _deps() + [os.path.join(CSRC, s) for s in SOURCES]
                 + [os.path.abspath(__file__)])
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= newest:
        return LIB
    nvcc = _nvcc()
    procs = []
    objs = []
    for src in SOURCES:
        obj = os.path.join(BUILD, src.replace('.cu', '.o'))
        objs.append(obj)
        cmd = [nvcc] + NVCC_FLAGS + ['-c', os.path.join(CSRC, src), '-o', obj]
        if verbose:
            print(' '.join(cmd))
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    errors = []
    for src, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            errors.append('%s:\n%s' % (src, out.decode(errors='replace')))
    if errors:
        raise RuntimeError('nvcc failed:\n' + '\n'.join(errors))
    tmp = LIB + '.%d.tmp' % os.getpid()
    subprocess.check_call([nvcc, '-shared', '-gencode', 'arch=compute_103a,code=sm_103a', '-o', tmp] + objs)
    os.replace(tmp, LIB)
    return LIB


if __name__ == '__main__':
    print(build(verbose=True))
