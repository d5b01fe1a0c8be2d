"""EXCMG + 19-point fourth-order compact scheme for the 3D Poisson equation on GB300.

The compute path lives in the CUDA library ``libexcmg.so`` (C-ABI declared in
``include/excmg.h``); ``paper_1507_05063_gb300.excmg`` is its thin ctypes binding and
``paper_1507_05063_gb300.autograd`` the torch.autograd wrapper around the adjoint.
``paper_1507_05063_gb300.problems`` holds the seeded closed-form input generators.
Importing this package loads nothing; importing ``.excmg`` loads the library and raises
if it has not been built.
"""
