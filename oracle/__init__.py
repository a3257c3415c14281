"""Plain FP64 CPU oracle of the symmetric Gauss-Seidel projection method (SGSPM).

This package is TEST INFRASTRUCTURE. It exists to check the CUDA path, and only
`tests/`, `__graft_entry__.smoke()` and the `cpu_baseline` / `--impl reference`
legs of `bench.py` may import or run it. The product path (the C-ABI library and
its Python binding) never calls into it, and the two share no code.

Modules
-------
newell   Newell demagnetising tensor of a uniform cell grid (analytic near field,
         Gauss-Legendre quadrature of the cell-pair dipole average in the far field).
demag    Stray field h_s = -N * m by zero-padded FFT and by brute-force summation.
heat     Implicit heat solve (I - c dt Delta_h)^{-1} by DCT-II/III, the mirror-ghost
         7-point Laplacian, and a dense LU solve of the assembled matrix.
scheme   Effective field, the SGSPM step (Sec. 3.2), the GSPM step (Sec. 3.1), the
         discrete energy and the manufactured solutions of Sec. 5.1.
spectral Spectral radii of the GS and SGS iteration matrices of a step (Sec. 4), from the
         intermediates of an oracle step (block reading stated there; parity with Tables 1-2
         unpinned).

Everything is float64 numpy/scipy; every function cites the passage it follows.
"""
