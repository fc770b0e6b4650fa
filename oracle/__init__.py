"""CPU oracle for the DPLR long-range hot path (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import, call, link or execute anything in this package.  The
product path (the CUDA library and its Python binding) never touches it, and
the two share no code: each side implements the method from the paper on its
own.  The only shared module is the seeded input generator in ``workloads/``,
which holds none of the method's arithmetic.

Contents:
  ewald.c            direct FP64 sums: E_Gt of Eq. DPLR:EGt with forces and
                      virial, the real-space erfc sum of point-charge Ewald,
                      and a brute-force erf image-shell sum.
  influence.c        the optimal ik influence function as plain loops.
  native.py          ctypes wrapper that compiles and loads the two C files.
  pppm.py             plain FP64 PPPM (Poisson-ik) with numpy.
  mlp.py              FP64 features, forward/backward and Adam of the
                      coarse-mesh correction network.
  wc_fold.py          FP64 fold of WC forces onto atoms (Eq. DPLR:F_final).
  dft_quant.py        the DFT with int32-quantised per-node partial sums of
                      the paper's hardware-offloaded FFT, and the PPPM that
                      uses it for every transform.
"""
