"""B300-native Cholesky-decomposed J/K engine (sm_103a).

The compute path lives in ``libjk.so`` (CUDA C++, C ABI, see include/jk.h);
``paper_2608_06536_b300.jk`` is the thin ctypes binding and
``paper_2608_06536_b300.autograd`` the torch.autograd wrapper.  Importing
the package itself loads nothing, so the seeded input generators in
``paper_2608_06536_b300.inputs`` can be used without a GPU.
"""
__all__ = ["inputs", "jk", "autograd"]
