"""B300-native randUTV minimum-norm least-squares solver.

The compute path lives in the CUDA library ``liblls.so`` (sources in
``csrc/``); ``lls`` is its thin ctypes binding and ``workloads`` draws the
seeded synthetic inputs.  Submodules are imported on demand so that the
input generators can be used without loading the library.
"""
