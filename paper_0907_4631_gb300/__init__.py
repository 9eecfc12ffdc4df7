"""GB300-native phipm: adaptive time-stepped Krylov evaluation of
u(t) = sum_k t^k phi_k(tA) b_k (Niesen & Wright, Sec. 3) on sm_103a."""
