// presplit.h -- host pre-split of fiber segments (see presplit.cpp).
#pragma once
#include <array>
#include <cstdint>
#include <vector>

namespace fx {

struct PieceRec {
  float pdt[16];  // (p, d, t0, t1) x (x, y, z, r), world space
  float root_radius;  // conservative radius of the piece's bounding cylinder (Sec. 3.3)
  float bound_radius; // sphere about the chord midpoint holding the root node's capped
                      // cylinder (+inf when an end plane does not bound it)
  int32_t level;  // pre-split level k (the piece is [off, off + 1] * 2^-k)
  int32_t off;
  bool unsupported;
};

// Pieces of all segments in segment order; begin[s] .. begin[s + 1] are the
// pieces of segment s (begin has n_seg + 1 entries).
// cps: n_seg x 4 control points x (x, y, z, r), in double precision.
void presplit_all(const double* cps, int64_t n_seg, int max_level, bool thick, int n_threads,
                  std::vector<PieceRec>& pieces, std::vector<int32_t>& begin);

}  // namespace fx
