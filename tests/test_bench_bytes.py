"""The benchmark's algorithmic byte count of one solve, on a hand-worked case.

Case: nnzb = 10 blocks of 1 x 1, n = 4 unknowns, S = 3 shifts, mixed
precision (FP32: 8 B per complex unknown, 8 B per complex value), 3
multi-shift iterations with shift 0 the base (met tol at iteration 3),
shift 1 at iteration 2, shift 2 at iteration 1; one reliable update in the
stage; one refinement round over shifts 1 (2 iterations) and 2 (1).

  matrix = 10 * (8 + 4) = 120 B; SpMV = 120 + 2 * 4 * 8 = 184 B
  FP64 residual = 10 * (16 + 4) + 2 * 4 * 16 + 4 * 16 + 4 * 8 = 424 B
  iteration 1: update 3 + 2 + 4 (shift 1) + 3 (shift 2, last) = 12 passes,
               184 + (3 + 12) * 32 = 664
  iteration 2: 3 + 2 + 3 (shift 1, last) = 8 passes: 184 + 11 * 32 = 536
  iteration 3: 5 passes: 184 + 8 * 32 = 440                 stage: 1640
  reliable update + final fold: 2 folds * 3 shifts * 40 B * 4 + 1 * 424 = 1384
  checks: (3 + 2 refined) * 424 = 2120
  refinement: k = 1, two shifts: 120 + 2 * 10 * 32 = 760;
              k = 2, one shift: 120 + 10 * 32 = 440            = 1200
  total 6344 B.
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


class _Info:
    iters = 3
    shift_iters = np.array([3, 2, 1])
    reliable_updates = 1
    refine_reliable_updates = 0
    refine_rounds = 1
    shift_refine_iters = np.array([0, 2, 1])


def test_solve_bytes_hand_worked_case():
    assert bench.solve_bytes(_Info(), 3, 10, 1, 4, mixed=True) == 6344


def test_spmv_bytes_of_the_benchmark_operator():
    # 24^4 block-CSR: 10,948,608 blocks of 3 x 3, 995,328 unknowns, FP32
    assert bench.spmv_bytes(10948608, 3, 995328, 4) == 848019456


class _StagInfo:
    """Two right-hand sides x two shifts on the stencil path (see below)."""
    iters = 3
    shift_iters = np.array([[3, 1], [2, 1]], dtype=np.int32)
    reliable_updates = 2
    refine_reliable_updates = 1
    refine_rounds = 1
    shift_refine_iters = np.array([[0, 2], [0, 0]])


def test_stencil_solve_bytes_hand_worked_case():
    """V = 16 sites of SU(3), two-row FP32 links, mixed: u = 24 B per site
    vector, l = 4 * 6 * 8 = 192 B of FP32 links and l64 = 4 * 9 * 16 = 576 B
    of FP64 links per site; one FP64 residual = 2 * 576 + 2 * 48 + 3 * 48 +
    24 = 1416 B per site.
      RHS 0: k = 1 update 5 + 3 = 8 passes -> 16 * (2 + 4 + 8) * 24 = 5376;
             k = 2, 3: 16 * 11 * 24 = 4224 each               = 13824
      RHS 1: 5376 + 4224                                        =  9600
      links of both passes, 3 iterations: 3 * 2 * 16 * 192     = 18432
      folds (1 reliable update + the final one per RHS) x 2 shifts x 40 * 3 * 16
                                                                = 11520
      the stage's reliable update: FP64 residual 16 * 1416      = 22656
      the refinement's reliable update: FP64 residual 22656 + the
      fold of its one shift 40 * 3 * 16 = 1920                  = 24576
      checks (4 + 1 refined) * 16 * 1416                        = 113280
      refinement k = 1, 2: 2 * 16 * 192 + 16 * 11 * 24 each     = 20736
      total 234624 B."""
    assert bench.stencil_solve_bytes(_StagInfo(), 2, 16, 3, 1, mixed=True) == 234624
