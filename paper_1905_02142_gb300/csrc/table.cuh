// Cubic-Hermite interpolation of the radial table (mixed-precision path).
//
// Node k (r_k = k h) holds two half-nodes of TableDims::FP floats: the values, then h times
// the r-derivatives.  Within a half-node the NC radial coefficients b_n come first, padded
// to a multiple of 4, then the LC + 1 angular factors 4 pi ilexp_l, also padded to 4, so that
// both groups are read with 16-byte loads.  Node k + 1 follows node k directly: the two
// nodes of an interval are 4 FP contiguous floats.
#pragma once
#include "internal.h"

template <int NC, int LC> struct TableDims {
  static constexpr int NCP = (NC + 3) / 4 * 4;      // b_n slots
  static constexpr int LPP = (LC + 1 + 3) / 4 * 4;  // ilexp_l slots
  static constexpr int FP = NCP + LPP;              // floats per half-node
};

// Interval of r: node index k (the interval [r_k, r_k+1], clamped to the table) and the
// fraction t of the way through it.
__device__ __forceinline__ int table_locate(const TableInfo& ti, float r, float& t) {
  const float x = r * ti.inv_h;
  int k = (int)x;
  k = k < 0 ? 0 : (k >= ti.K ? ti.K - 1 : k);
  t = x - (float)k;
  return k;
}

// Cubic-Hermite interpolation from the 4 FP floats of one interval (nodes k and k + 1),
// in global memory (GLOBAL: read-only loads) or in a shared-memory copy (STREAM: four slots
// at a time, fewer live registers; otherwise the whole interval is loaded first):
// f[0..NC) = b_n(r), f[NC..NC+LC] = 4 pi ilexp_l(r); df = d/dr of the same (if DERIV).
template <int NC, int LC, bool DERIV, bool GLOBAL = false, bool STREAM = false>
__device__ __forceinline__ void table_interp_at(const float4* __restrict__ n0, float t, float invh, float* f,
                                                float* df) {
  using TD = TableDims<NC, LC>;
  constexpr int Q = TD::FP / 4;  // float4 per half-node
  const float t2 = t * t;
  const float h00 = (2.f * t - 3.f) * t2 + 1.f, h10 = ((t - 2.f) * t + 1.f) * t;
  const float h01 = (3.f - 2.f * t) * t2, h11 = (t - 1.f) * t2;
  const float d00 = 6.f * t * (t - 1.f), d10 = (3.f * t - 4.f) * t + 1.f, d11 = (3.f * t - 2.f) * t;
  auto out = [&](int j, float a0, float b0, float a1, float b1) {
    int o;  // logical output index, or -1 for a padding slot
    if (j < TD::NCP) o = j < NC ? j : -1;
    else o = (j - TD::NCP) <= LC ? NC + (j - TD::NCP) : -1;
    if (o < 0) return;
    f[o] = h00 * a0 + h10 * b0 + h01 * a1 + h11 * b1;
    if (DERIV) df[o] = (d00 * (a0 - a1) + d10 * b0 + d11 * b1) * invh;
  };
  if constexpr (!STREAM) {
    // the whole interval first (all loads in flight together)
    float4 v0[Q], g0[Q], v1[Q], g1[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      if constexpr (GLOBAL) {  // read-only path
        v0[q] = __ldg(n0 + q);
        g0[q] = __ldg(n0 + Q + q);
        v1[q] = __ldg(n0 + 2 * Q + q);
        g1[q] = __ldg(n0 + 3 * Q + q);
      } else {
        v0[q] = n0[q];
        g0[q] = n0[Q + q];
        v1[q] = n0[2 * Q + q];
        g1[q] = n0[3 * Q + q];
      }
    }
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      out(4 * q + 0, v0[q].x, g0[q].x, v1[q].x, g1[q].x);
      out(4 * q + 1, v0[q].y, g0[q].y, v1[q].y, g1[q].y);
      out(4 * q + 2, v0[q].z, g0[q].z, v1[q].z, g1[q].z);
      out(4 * q + 3, v0[q].w, g0[q].w, v1[q].w, g1[q].w);
    }
  } else {
    static_assert(!GLOBAL, "streamed interpolation reads shared memory");
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const float4 v0 = n0[q], g0 = n0[Q + q], v1 = n0[2 * Q + q], g1 = n0[3 * Q + q];
      out(4 * q + 0, v0.x, g0.x, v1.x, g1.x);
      out(4 * q + 1, v0.y, g0.y, v1.y, g1.y);
      out(4 * q + 2, v0.z, g0.z, v1.z, g1.z);
      out(4 * q + 3, v0.w, g0.w, v1.w, g1.w);
    }
  }
}

// The same, reading the interval of r from the table in global memory.
template <int NC, int LC, bool DERIV>
__device__ __forceinline__ void table_interp(const float* __restrict__ tab, const TableInfo& ti,
                                             float r, float* f, float* df) {
  constexpr int Q = TableDims<NC, LC>::FP / 4;
  float t;
  const int k = table_locate(ti, r, t);
  const float4* n0 = reinterpret_cast<const float4*>(tab) + (size_t)k * 2 * Q;
  table_interp_at<NC, LC, DERIV, true>(n0, t, ti.inv_h, f, df);
}
