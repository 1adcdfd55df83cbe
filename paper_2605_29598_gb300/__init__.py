"""GB300-native hot path of a rotating IMEX-DG solver for the compressible
Euler equations (matrix-free DG on quad/hex meshes with 2:1 hanging faces).

The compute path lives in ``libdgimex.so`` (CUDA, sm_103a) behind a C ABI
declared in ``include/dgimex.h``; :mod:`.dgimex` is its ctypes binding and
:mod:`.inputs` builds synthetic meshes and initial states.  Importing this
package loads nothing: the shared library is opened on first use.
"""
__all__ = ["inputs", "dgimex"]
