// Device helpers of the row kernels (ham.cu): two-body table lookups and the
// double-float value sums.  Not part of the ABI.
#pragma once

#include <cstdint>

#include "cih_internal.h"

namespace cih {

// Table layout caps of the shared-memory copies the kernels keep.
constexpr int kLayoutCap = 512;   // global table groups
constexpr int kOrbCap = 512;      // combined orbitals (two species of at most 256)
constexpr int kGroupCap = 128;    // dense pn group keys

// Table index of V(ab, cd) for combined orbitals in any order; false if the
// pairs are not one table entry (a bug in the walk: flagged by the caller).
// The group sizes and offsets come from shared memory (lg: size and offset
// per group, int2) when the layout has at most kLayoutCap groups.
__device__ __forceinline__ bool tbme_at(const DevBasis &B, const int2 *lg, int a, int b, int c, int d, int64_t &idx,
                                        int &sign)
{
    if ((unsigned)a >= (unsigned)B.ntot || (unsigned)b >= (unsigned)B.ntot ||
        (unsigned)c >= (unsigned)B.ntot || (unsigned)d >= (unsigned)B.ntot)
        return false;
    int32_t e1 = B.pid[a * B.ntot + b], e2 = B.pid[c * B.ntot + d];
    if (e1 < 0 || e2 < 0) return false;
    int g = (e1 >> 16) & 0xFFF;
    if (g != ((e2 >> 16) & 0xFFF)) return false;
    sign = (((e1 ^ e2) >> 30) & 1) ? -1 : 1;
    int u = e1 & 0xFFFF, v = e2 & 0xFFFF;
    if (u > v) { const int t = u; u = v; v = t; }
    int64_t n, off;
    if (B.ngroups <= kLayoutCap) {
        const int2 q = lg[g];
        n = q.x;
        off = q.y;
    } else {
        n = B.gsize[g];
        off = B.goff[g];
    }
    idx = off + (int64_t)u * n - (int64_t)u * (u - 1) / 2 + (v - u);
    return true;
}

// A sum of FP32 terms carried as the unevaluated pair hi + lo of floats
// (Dekker's two-sum), about 48 significant bits: exact for the value sums here
// (at most a few dozen FP32 terms within 24 binary orders of magnitude), and
// single-precision arithmetic runs at full rate where the GPU's FP64 units are
// few.  The value stored is hi + lo rounded once to FP32.
struct DF {
    float hi, lo;
};
__device__ __forceinline__ DF df_add(DF a, DF b)
{
    const float s = a.hi + b.hi;
    const float bb = s - a.hi;
    const float e = (a.hi - (s - bb)) + (b.hi - bb);
    const float lo = (e + a.lo) + b.lo;
    const float hi = s + lo;
    return DF{hi, lo - (hi - s)};
}
__device__ __forceinline__ DF df_of(float x) { return DF{x, 0.f}; }
__device__ __forceinline__ float df_round(DF v) { return v.hi + v.lo; }

// table index of a pn element from the candidate (uv, mv) and neutron move (ni):
// u(a, b) = S[a][kappa] + r(b), v(c, d) = S[c][kappa] + r(d), kappa the dense
// (2M_pair, parity) key; sign = proton move sign ^ neutron move sign
__device__ __forceinline__ int pn_index_at(const int16_t *S, const int32_t *gs, const int32_t *go, uint32_t uv,
                                           uint32_t mv, uint32_t ni, int &sign)
{
    const int t = (int)((ni >> 16) & 0x7F) - 64 + (int)(((mv >> 8) ^ (ni >> 23)) & 1);
    const int kappa = (int)(mv & 0xFF) + t;
    int u = S[(int)(uv & 0xFFFF) + t] + (int)((ni >> 8) & 0xFF);
    int v = S[(int)(uv >> 16) + t] + (int)(ni & 0xFF);
    if (u > v) { const int x = u; u = v; v = x; }
    sign = (int)(((mv >> 9) ^ (ni >> 24)) & 1);
    return go[kappa] + u * gs[kappa] - ((u * (u - 1)) >> 1) + (v - u);
}

}  // namespace cih
