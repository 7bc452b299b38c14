"""CPU FP64 oracle for contraction-tree execution (arXiv 2002.01935).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the package smoke check
and by the CPU-baseline leg of the benchmark.  The product path never imports
it; it imports nothing from the product package.

  oracle.tree        -- FP64/complex128 tree executor (C, explicit loop nests)
  oracle.brute       -- the nested sum of products, written out (Sec. 4.7.1)
  oracle.statevector -- dense state-vector simulation of circuits (Eq. trans-amp)
  oracle.ising       -- partition functions by enumeration and closed forms
  oracle.gradient    -- leaf derivatives as environment contractions
"""
