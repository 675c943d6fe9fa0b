// hydro_uniform.cuh -- the work list of a uniform batch computed on the
// device from its sub-grid descriptors (used by hydro_rhs_ex, which builds
// such lists with a small kernel, and by the allocation-free entry point,
// whose tile kernel reads the descriptors directly).
#pragma once

#include "hydro.h"
#include "hydro_kernels.cuh"

namespace hydro_dev {

// Tile t of a uniform batch (one N, one field count) computed from the
// sub-grid descriptors: sub-grid t / tps, tile t % tps of it in x-fastest
// order.  The same fields, with the same arithmetic (an IEEE division for
// 1/dx; the power-of-two test on the bit pattern), as the host's work list.
struct UniformDesc {
  const hydro_subgrid_t* __restrict__ desc;
  int N, F, G, tpe;  // tpe: tiles per edge
  __device__ __forceinline__ Tile operator()(int t) const {
    const int tps = tpe * tpe * tpe;
    const int s = t / tps, k = t - s * tps;
    const hydro_subgrid_t d = desc[s];
    Tile tile;
    tile.U = d.U;
    tile.out_off = (long long)s * F * N * N * N;
    tile.amax_off = s;
    tile.inv_dx = 1.0 / d.dx;
    tile.sub = s;
    tile.N = N;
    tile.F = F;
    tile.G = G;
    tile.ox = (short)((k % tpe) * TE);
    tile.oy = (short)(((k / tpe) % tpe) * TE);
    tile.oz = (short)((k / (tpe * tpe)) * TE);
    // dx an exact power of two (frexp mantissa 1/2, exponent within +-120)
    long long b = __double_as_longlong(d.dx);
    int e2 = (int)((b >> 52) & 0x7ff) - 1022;
    bool pow2 = (b & 0x000fffffffffffffLL) == 0 && ((b >> 52) & 0x7ff) != 0 && e2 > -120 && e2 < 120;
    tile.flags = (short)((tps > 1 ? 1 : 0) | (pow2 ? 2 : 0));
    tile.pad[0] = tile.pad[1] = 0;
    return tile;
  }
};

}  // namespace hydro_dev
