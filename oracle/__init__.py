"""Plain FP64 CPU oracle for the chi0 / W hot path of RESPACK (arXiv 2001.02351).

TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU
baseline leg of the benchmark may import this package; the library under
`paper_2001_02351_gb300/` never does, and this package never imports it.
It shares no code, table or helper with the CUDA path; the only common
module is the seeded input generator `synth/`, which holds none of the
method's arithmetic.

Each function follows the paper's statement of the method:
  lattice.py       -- sphere cut-offs (Eq. pak, Sec. 2.3 epsilon sphere),
                      umklapp map k+q = k' + G0
  pair_density.py  -- M^G_ab(k+q,k) by direct G-space convolution (Eq. ism)
  tetra.py         -- generalized-tetrahedron weights x(k) (Eq. tetrahedron)
                      and the plain Lorentzian X (Eq. Xakqbk)
  chi0.py          -- chi_GG'(q,w) dense sum (Eq. chi)
  dyson.py         -- symmetric epsilon (Eq. epsGG), W (Eq. Wq)
  freqgrid.py      -- logarithmic frequency grid (Eq. grid)

Parity status: every function is pinned by tests under tests/ (closed forms,
invariants, brute force) except the tetrahedron scheme's agreement with the
exact published Fujiwara/Nohara implementation, which the paper does not
print: the oracle pins its own stated reading of that scheme (parity
unpinned against the published code).
"""
