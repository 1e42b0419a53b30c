"""CPU oracle for the GSGP hot path: test infrastructure, not product code.

A plain, slow and deliberately unoptimised float64 restatement of Geometric
Semantic GP for symbolic regression (Trujillo et al., "GSGP-CUDA", Sec. 2 and
Algorithm 1).  It exists only so that the tests, the smoke check and the CPU
baseline leg of the benchmark can check and time the CUDA library against an
independent implementation.  It shares no code, header, table or constant
generator with the CUDA path and never imports it; the CUDA library never
imports, links or calls anything here.

Modules:
  philox  - Philox4x32-10 (Salmon et al., SC'11) and the integer-only mappings
            from random words to indices, uniforms and constants.
  trees   - ramped half-and-half postfix program generation (initialisation).
  interp  - postfix stack interpreter and an independent recursive evaluator
            (the ComputeSemantics step), logistic wrapping of random trees.
  gsgp    - fitness (RMSE), tournament selection, geometric semantic mutation,
            survival with elitism, the ancestry trace, reconstruction and
            prediction of the best individual; independent and replay modes.
"""
