"""Algorithmic FP32 work of the traversal, per counted event.

Counts follow the arithmetic of each step as the kernels perform it (an add,
subtract or multiply is one flop, a fused multiply-add two, a reciprocal,
division or square root one); comparisons, selects and integer bit-string
work are not counted.  Work that only some events need is not charged (the
slab and the rotation of t0, t1 that a passing root cylinder needs), so the
totals are lower bounds.

  per ray          normalise the direction, Duff et al.'s basis          20
  per candidate    origin offset, ray-frame z of p and d, the bound of
                   the root node's capped cylinder against t_max          20
  per root node    x, y of p and d in the ray frame (20) + unit-ray
                   cylinder with the precomputed root radius (24)         44
  per deeper node  conservative radius (44) + unit-ray cylinder (24)      68
  per descent      split terms, plane, child selection                    49
  per backtrack    power-form recomputation (142) + slab (15)            157
  per hit          u by projection onto the leaf axis, segment mapping    17

The paper's algorithm performs more for the same frame: it has no bound
test, so every candidate pays the setup of Sec. 3.1 / 3.3 and a root node
test like any node (method_flops):

  per candidate    four control points into the ray frame (4 x 18),
                   (p, d, t0, t1) differences (12), end-plane slab (15)   99
                   + root node test as a deeper node                      68

Descents, backtracks and hits are the same events on both: the bound test
only removes root tests that cannot pass.

A third, coarser count takes per-unit estimates from the operation counts
of App. C's routines instead of the kernels' arithmetic (estimate_flops),
for the paper's algorithm on the same events:

  per ray with candidates   ONB: about 12 operations + 1 reciprocal      13
  per candidate             setup of Sec. 3.1 / 3.3                      75
  per node test             test and partition/descent: about 120 flops
                            + 3 reciprocals + 2 square roots (every
                            candidate's root tested as a node)          125
  per backtrack             recomputation: 105 operations + 2 rcp        107
  per hit                   final: 12 operations + 1 division            13

Counters (all variants): tests = candidate pieces examined, nodes = node
tests including roots, descents, backtracks, hits.  Every deeper node test
follows a descent or a backtrack, so root node tests = nodes - descents -
backtracks.
"""

PER_RAY = 20
PER_BOUND = 20
PER_ROOT = 44
PER_NODE = 68
PER_DESCENT = 49
PER_BACKTRACK = 157
PER_HIT = 17

PER_SETUP_METHOD = 99

EST_RAY = 13
EST_SETUP = 75
EST_NODE = 125
EST_BACKTRACK = 107
EST_HIT = 13

# Bytes a closest-hit launch must move at least once: ray (32 B) and two
# row_ptr words per ray, one seg_idx word per pair, 64 B per piece touched,
# 16 B of output per ray (tu, seg, leaf).
BYTES_PER_RAY = 32 + 8 + 16
BYTES_PER_PAIR = 4
BYTES_PER_PIECE = 64


def alg_flops(counters, n_ray_with_candidates):
    c = counters
    deeper = c["descents"] + c["backtracks"]
    return (PER_RAY * n_ray_with_candidates + PER_BOUND * c["tests"] + PER_ROOT * (c["nodes"] - deeper)
            + PER_NODE * deeper + PER_DESCENT * c["descents"] + PER_BACKTRACK * c["backtracks"]
            + PER_HIT * c["hits"])


def method_flops(counters, n_ray_with_candidates):
    """The paper's algorithm on the same frame: every candidate set up and
    its root tested as a node, then the same descents, backtracks and hits."""
    c = counters
    deeper = c["descents"] + c["backtracks"]
    return (PER_RAY * n_ray_with_candidates + (PER_SETUP_METHOD + PER_NODE) * c["tests"] + PER_NODE * deeper
            + PER_DESCENT * c["descents"] + PER_BACKTRACK * c["backtracks"] + PER_HIT * c["hits"])


def estimate_flops(counters, n_ray_with_candidates):
    """The paper's algorithm on the same events, with the per-unit estimates
    from the operation counts of App. C (see the module docstring)."""
    c = counters
    deeper = c["descents"] + c["backtracks"]
    return (EST_RAY * n_ray_with_candidates + EST_SETUP * c["tests"] + EST_NODE * (c["tests"] + deeper)
            + EST_BACKTRACK * c["backtracks"] + EST_HIT * c["hits"])


def alg_bytes(n_ray, n_pair, n_piece_touched):
    return BYTES_PER_RAY * n_ray + BYTES_PER_PAIR * n_pair + BYTES_PER_PIECE * n_piece_touched


def fp32_peak_tflops(sm_count, sm_mhz):
    """FP32 FMA peak: 128 lanes per SM, 2 flops per FMA."""
    return sm_count * 128 * 2 * sm_mhz * 1e6 / 1e12
