// slot_map.cuh -- where the guard cells of a block's neighbour slot come
// from, as a linear map of padded cell coordinates; shared by the fused tile
// load (hydro_tile.cuh) and the same-level guard copy (grid_ops.cuh).
//
// Paper: Flash-X (arXiv 2208.11630), Section 2 -- the Grid unit fills guard
// cells from same-level neighbours and applies the physical boundaries.
#pragma once

#include "fx_internal.h"

namespace fx {
namespace {

// Where the guard cells of slot q (= sx + 3 sy + 9 sz, with 1 = the block's
// own range on that axis) of block b come from, as a map that is linear in the
// padded cell coordinates (gx, gy, gz) of b: the cell's first variable sits at
// element off + gx c.x + gy c.y + gz c.z of the state array, and bit d of c.w
// says that the d velocity component is mirrored.  A same-level slot reads
// the neighbour's interior (per axis a shift, the periodic wrap included); at
// a physical boundary an outflow axis clamps to the edge cell (coefficient 0)
// and a reflecting axis mirrors (coefficient -1, velocity negated).  Slots
// covered by a coarser leaf, and the block's own cells, map to the block's
// own padded array.
__device__ __forceinline__ void guard_source(const DevMesh &m, int b, int q, long long &off,
                                             int4 &c) {
  const int2 sl = m.slots[b * 27 + q];
  const int P = m.P, ng = m.ng, n = m.nxb, lev = m.level[b];
  const bool copy = q != 13 && sl.x == SLOT_COPY;
  const int src = copy ? sl.y : b;
  int coef[3] = {1, 1, 1}, k[3] = {0, 0, 0};
  unsigned flip = 0;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    if (!copy || d >= m.ndim) continue;
    const int sd = d == 0 ? q % 3 : (d == 1 ? (q / 3) % 3 : q / 9);
    const int o = m.origin[3 * b + d], os = m.origin[3 * src + d], N = m.ncell[lev][d];
    // padded index in the source = index in the level lattice - os + ng;
    // the block's own cell gx sits at lattice index o + gx - ng
    k[d] = o - os;
    if (sd == 1) continue;
    const bool lo = sd == 0;
    if (lo ? o != 0 : o + n < N) continue;   // inside the domain
    const int kind = m.bc[d][lo ? 0 : 1];
    if (kind == FX_BC_PERIODIC) {
      k[d] = lo ? o + N - os : o - N - os;
    } else if (kind == FX_BC_REFLECT) {
      // lattice index -1 - a (low side) or 2N - 1 - a (high side)
      coef[d] = -1;
      flip |= 1u << d;
      k[d] = (lo ? -1 : 2 * N - 1) - o + 2 * ng - os;
    } else {
      // outflow: the edge cell, 0 or N - 1
      coef[d] = 0;
      k[d] = (lo ? 0 : N - 1) + ng - os;
    }
  }
  off = (long long)src * m.bstride + ((long long)k[2] * P + k[1]) * P + k[0];
  c = make_int4(coef[0], coef[1] * P, coef[2] * P * P, (int)flip);
}

}  // namespace
}  // namespace fx
