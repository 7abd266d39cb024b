"""libkrr: GB300-native preconditioned Krylov solvers for Gaussian-kernel
regression (flexible GMRES right-preconditioned by truncated CG on the more
strongly regularised kernel matrix)."""
