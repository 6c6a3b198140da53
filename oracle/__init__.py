"""CPU oracle of the TTIE hot path.

TEST INFRASTRUCTURE ONLY.  Plain, slow FP64 (and exact rational) restatement
of "Differentiable 3D Triangle-Triangle Intersection Energy" used to check the
CUDA path.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import it; the library never does, and it shares no
code with the CUDA kernels.

Parity status of each function:
  pair_dual.c oracle_pair    pinned: closed-form pairs (Eq. 1-2), central
                             finite differences, invariances
  exact.active_exact         pinned: independent separating-axis brute force
                             on integer-grid triangle pairs
  pair_dual.c filtered_side  pinned: agrees with exact signs on random and
                             near-degenerate inputs
  gradient / hessian_*       pinned: FD of T, closed-form eigenvalues (§1.1),
                             sympy derivation of the dropped Eq. 4 terms
  hessian_vector_product     pinned: Euler's identity H x = 3 g (T has degree 4),
                             H (w x x) = w x g (rotation invariance), H 1 = 0
                             (translation), v.Hv = second difference of E
  assemble / newton_solve    pinned: dense recomputation, direct solve
                             residual, the line-search rule on a quadratic
                             whose decisions are known, the step cap; the
                             Newton trajectory itself is parity-unpinned
                             (only the certified end state is compared)
  elastic.*                  pinned: spring closed forms, central finite
                             differences, projected-spectrum closed form,
                             invariances (the elastic model is a reading: the
                             paper does not state it)

The pins are themselves checked: tests/test_oracle_mutations.py plants one
plausible mistake at a time in a copy of this package and requires the pin
that covers it to fail.
"""
from .ttie_oracle import (build_oracle, candidate_pairs, partners_of, evaluate,  # noqa: F401
                          eval_pairs_f64, filtered_sides, gradient, hessian_parts,
                          hessian_inexact, hessian_psd, clamp_psd, assemble, pair_dofs,
                          blocks_to_dense, hessian_vector_product, pair_hessian_vector,
                          newton_direction, newton_solve, line_search, next_overshoot, capped_direction,
                          certify, energy,
                          NewtonParams, PairEval)
from . import exact  # noqa: F401
from .elastic import (Elastic, mesh_edges, springs_at_rest, elastic_energy, elastic_gradient,  # noqa: F401,E402
                      spring_hessian, elastic_blocks, elastic_vertices, total_energy,
                      newton_direction_elastic, quasi_static_solve)
