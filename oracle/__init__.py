"""CPU FP64 oracle for the phipm method (Niesen & Wright, Sec. 2-3).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
link anything under this package: only the tests, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` use it.  It shares no code with the
CUDA implementation; the two meet only at the seeded input generators in
``paper_0907_4631_gb300.workloads``, which hold no arithmetic of the method.

Modules:
  phipm_oracle  the algorithm itself (Algorithms 1-4, Eqs. phipapprox2, errest,
                step, wrecurrence, tau_0, taunew, 2, 3, 4, 5, 6, 7, 8)
  truth         exact answers independent of the algorithm (closed forms of
                phi_k, the sine eigen-expansion of the Dirichlet Laplacian,
                dense exponential of the augmented matrix)
  mlp_oracle    FP64 forward/backward of the learned (tau, m) controller network
"""
