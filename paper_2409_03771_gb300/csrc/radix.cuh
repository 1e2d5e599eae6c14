// Device helpers shared by the radix-sort kernels of the vertex order
// (Simulation of Simplicity, section "Preprocessing": sort by value, ties
// by global id) and of the 64-bit pair sorts.
#pragma once

#include "common.cuh"

namespace msc {

constexpr int kRadixBins = 256;      // 8-bit digits
constexpr int kRadixScanWarps = 8;   // warps of the 256-thread blocks that scan

// float32 bits -> an unsigned key with the same order (IEEE '<'); -0.0 is
// first folded onto +0.0 so that the two tie.
__device__ __forceinline__ uint32_t float_key(float x) {
    uint32_t u = __float_as_uint(x);
    if (u == 0x80000000u) u = 0u;  // -0.0 ties with +0.0
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ bool is_nan_bits(float x) {
    return (__float_as_uint(x) & 0x7fffffffu) > 0x7f800000u;
}

// Inclusive scan over 256 values held one per thread of a 256-thread block
// (s_w: 8 words of shared scratch).
__device__ __forceinline__ uint32_t block_scan_256(uint32_t v, uint32_t* s_w) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    if (lane == 31) s_w[warp] = v;
    __syncthreads();
    if (warp == 0) {
        uint32_t t = lane < kRadixScanWarps ? s_w[lane] : 0u;
#pragma unroll
        for (int o = 1; o < kRadixScanWarps; o <<= 1) {
            const uint32_t q = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += q;
        }
        if (lane < kRadixScanWarps) s_w[lane] = t;
    }
    __syncthreads();
    if (warp > 0) v += s_w[warp - 1];
    __syncthreads();
    return v;
}

// Lanes of the warp whose 8-bit digit equals this lane's (valid lanes
// only), from eight ballots -- no match instruction, no divergence.
__device__ __forceinline__ uint32_t digit_peers(uint32_t d, bool valid) {
    uint32_t eq = __ballot_sync(0xffffffffu, valid);
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        const bool bit = (d >> b) & 1u;
        const uint32_t bal = __ballot_sync(0xffffffffu, bit);
        eq &= bit ? bal : ~bal;
    }
    return eq;
}

// The same for a warp whose 32 lanes all hold a valid digit.
__device__ __forceinline__ uint32_t digit_peers_all(uint32_t d) {
    uint32_t eq = 0xffffffffu;
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        const bool bit = (d >> b) & 1u;
        const uint32_t bal = __ballot_sync(0xffffffffu, bit);
        eq &= bit ? bal : ~bal;
    }
    return eq;
}

constexpr int kHistRun = 16;  // consecutive keys per thread in the histogram

// Loads the float keys f[i0 .. i0+cnt) (cnt <= 16; the rest become 0)
// into k[], noting NaNs.
__device__ __forceinline__ void load_float_keys16(const float* __restrict__ f, int64_t i0, int cnt,
                                                  uint32_t (&k)[kHistRun], bool& saw_nan) {
    if (cnt == kHistRun && ((uintptr_t)(f + i0) & 15) == 0) {
#pragma unroll
        for (int q = 0; q < kHistRun / 4; ++q) {
            const float4 v = reinterpret_cast<const float4*>(f + i0)[q];
            saw_nan |= is_nan_bits(v.x) | is_nan_bits(v.y) | is_nan_bits(v.z) | is_nan_bits(v.w);
            k[4 * q + 0] = float_key(v.x);
            k[4 * q + 1] = float_key(v.y);
            k[4 * q + 2] = float_key(v.z);
            k[4 * q + 3] = float_key(v.w);
        }
    } else {
#pragma unroll
        for (int j = 0; j < kHistRun; ++j) {
            const float x = j < cnt ? f[i0 + j] : 0.f;
            saw_nan |= j < cnt && is_nan_bits(x);
            k[j] = float_key(x);
        }
    }
}

// Adds the digits of k[0 .. cnt) for `npass` passes to the histograms h
// ([npass][256]), one shared atomic per run of equal digits.
template <typename KeyT>
__device__ __forceinline__ void count_runs(const KeyT (&k)[kHistRun], int cnt, int npass, uint32_t* h) {
    for (int p = 0; p < npass; ++p, h += kRadixBins) {
        uint32_t cur = (uint32_t)(k[0] >> (8 * p)) & 255u, run = 1;
#pragma unroll
        for (int j = 1; j < kHistRun; ++j) {
            if (j >= cnt) break;
            const uint32_t d = (uint32_t)(k[j] >> (8 * p)) & 255u;
            if (d == cur) {
                ++run;
            } else {
                atomicAdd(&h[cur], run);
                cur = d;
                run = 1;
            }
        }
        atomicAdd(&h[cur], run);
    }
}

// Adds the run-length counted digits of k[0 .. cnt) at bit `shift` to the
// histogram h[256]: one shared atomic per run of equal digits.
template <typename KeyT>
__device__ __forceinline__ void count_runs_at(const KeyT (&k)[kHistRun], int cnt, int shift, uint32_t* h) {
    uint32_t cur = (uint32_t)(k[0] >> shift) & 255u, run = 1;
#pragma unroll
    for (int j = 1; j < kHistRun; ++j) {
        if (j >= cnt) break;
        const uint32_t d = (uint32_t)(k[j] >> shift) & 255u;
        if (d == cur) {
            ++run;
        } else {
            atomicAdd(&h[cur], run);
            cur = d;
            run = 1;
        }
    }
    atomicAdd(&h[cur], run);
}

}  // namespace msc
