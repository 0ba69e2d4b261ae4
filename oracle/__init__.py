"""CPU oracle for FNO-EOM-CCSDT (arXiv 2509.14157) -- TEST INFRASTRUCTURE ONLY.

Plain, slow, FP64 NumPy/SciPy implementation of what the CUDA library computes:
restricted Hartree-Fock, MP2 natural orbitals and their truncation (FNO/XFNO),
the CCSDT amplitude equations (Eq. 5-7) and the IP/EA/DIP/DEA EOM-CCSDT
eigenproblems (Eq. 1-4), together with a Fock-space (determinant) definition
oracle and full-CI diagonalisation that pin it.

Only the test suite, `__graft_entry__.smoke()` and the CPU-baseline leg of
`bench.py` may import this package. The library under
`paper_2509_14157_gb300/` never imports, links or calls it, and this package
never imports the library; the two share only the seeded inputs of `synth`.

Parity status of each part is stated in the module headers; every function
carries the passage of the paper it follows.
"""
