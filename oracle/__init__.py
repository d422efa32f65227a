"""CPU FP64 oracle for J-TRLan -- test infrastructure only.

Plain, slow, obviously-correct numpy code that states what the CUDA path must
compute.  Only the tests, the smoke check and the CPU-baseline leg of the
benchmark may import it; the library itself never does, and the oracle shares no
code with it (it reads nothing from the package; its inputs are plain arrays).

Contents:
  jsym        -- J, the pair map y = J x*, the block form of A (Sec. 1, eqs. (1), (2), (4)),
                 dense and 4D-stencil operators written from their definitions, and
                 brute-force dense assembly for small problems.
  trlan_jsym  -- Algorithm 1 (TRLAN-JSYM) and Algorithm 2 (LANCZOS_JSYM) in FP64,
                 in the paper's order and notation.
  jacobi      -- the cyclic Jacobi eigensolver that diagonalises T_m in Algorithm 1.
  inertia     -- eigenvalue counts below a shift by Sylvester's law of inertia (LDL^H), which
                 check that Algorithm 1's nev pairs are the nev smallest.
  cg          -- conjugate gradients for the invert mode's products A^{-1} v.
  filter      -- polynomial filters p(A) (Chebyshev recurrence, damped step coefficients);
                 the paper has none, these are standard definitions.
  mlp         -- the 3-layer perceptron that predicts filter coefficients: forward pass,
                 gradient and one Adam step in FP64.
"""
