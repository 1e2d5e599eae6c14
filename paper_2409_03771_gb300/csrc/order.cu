// Vertex order (Simulation of Simplicity, section "Preprocessing": the
// vertices sorted by scalar value with ties broken by global id; order[v]
// is the position of v).
//
// LSD radix sort of (key, id) pairs, four 8-bit digit passes.  Keys are
// the float bits mapped to an order-preserving uint32 (-0.0 folded onto
// +0.0); every pass is stable and the first reads the vertices in id
// order, so equal keys stay in id order and the final position of v is its
// rank under (f[v], v).
//
// Each pass is an upsweep / scan / downsweep over super-tiles (runs of S
// consecutive 6144-key tiles), so no block ever waits for another:
//   k_ord_up    counts the pass digit of every super-tile (run-length
//               counted into warp-private shared histograms);
//   k_ord_scan  one block per digit turns the super-tile counts into each
//               super-tile's first output position for that digit;
//   k_ord_down  each block takes super-tiles s, s + G, s + 2G, ... (G
//               blocks), walks their tiles in order, ranks each tile's keys
//               stably (warp ballots), keeps running per-digit offsets and
//               writes through shared memory in coalesced runs.  The next
//               tile is fetched by a 1D TMA bulk copy into the other half
//               of a shared-memory double buffer while the current one is
//               ranked; the consumed half then serves as the staging area.
//               Interleaved super-tiles keep the blocks' write fronts of a
//               digit next to each other, so partly written lines are
//               completed in L2 before they are written back.
// The last pass files (vertex id, position) pairs into buckets of
// consecutive ids instead of writing sorted keys, and the order field is
// their inverse permutation (k_pair_split / k_pair_scatter_local).
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

#include "radix.cuh"
#include "sort.cuh"
#include "tma.cuh"

namespace msc {
namespace {

#ifndef MSC_ORD_ITEMS
#define MSC_ORD_ITEMS 24
#endif
#ifndef MSC_ORD_MIN_BLOCKS
#define MSC_ORD_MIN_BLOCKS 2
#endif
#ifndef MSC_ORD_MATCH_MAX
#define MSC_ORD_MATCH_MAX 64
#endif
constexpr int kT = 256;                // threads per block
constexpr int kI = MSC_ORD_ITEMS;      // keys per thread and tile
constexpr int kTile = kT * kI;  // keys per tile (6144)
static_assert(kI % 4 == 0, "digits are packed four to a word");
constexpr int kW = kT / kWarp;  // 8 warps
constexpr int kB = kRadixBins;  // 256 digits
constexpr uint32_t kWaitLimit = 1u << 22;  // mbarrier polls before giving up (~0.3 s)

static_assert(kRadixScanWarps == kW, "block_scan_256 expects 8 warps");
static_assert(kOrderMaxBuckets == kT, "one id bucket per thread");

// Super-tile s holds tiles [s * per_super, min(tiles, (s + 1) * per_super)).
struct Range {
    int64_t n;
    int64_t tiles;
    int64_t per_super;
    int supers;
};

// The 8-bit digit of a key at a compile-time bit offset (one byte permute).
template <int SHIFT>
__device__ __forceinline__ uint32_t digit_of(uint32_t k) {
    if constexpr (SHIFT == 0) return k & 255u;
    else if constexpr (SHIFT == 24) return k >> 24;
    else return __byte_perm(k, 0u, 0x4440u + SHIFT / 8);
}

// Upsweep: per-super-tile counts of the digit at SHIFT, stored digit-major
// (cnt[d * kOrderMaxSuper + s]), plus the pass totals (one atomic per block
// and digit).  FROM_F: the keys are made from the float field, whose NaNs
// are reported here.
template <bool FROM_F, int SHIFT>
__global__ void __launch_bounds__(kT) k_ord_up(const float* __restrict__ f, const uint32_t* __restrict__ keys,
                                               const Range r, uint32_t* __restrict__ cnt,
                                               uint32_t* __restrict__ total, int32_t* status) {
    __shared__ uint32_t sh[kW * kB];
    const int tid = threadIdx.x, warp = tid >> 5;
    uint32_t* wh = sh + warp * kB;
    bool nan = false;
    uint32_t mine = 0;  // this block's total of digit tid
    const bool vec = FROM_F || ((uintptr_t)keys & 15) == 0;
    constexpr int64_t kStep = (int64_t)kT * kHistRun;
    for (int s = blockIdx.x; s < r.supers; s += gridDim.x) {
        for (int i = tid; i < kW * kB; i += kT) sh[i] = 0;
        __syncthreads();
        const int64_t k0 = (int64_t)s * r.per_super * kTile;
        const int64_t k1 = min(r.n, k0 + r.per_super * kTile);
        // two groups of 16 consecutive keys per thread and step: both groups'
        // loads are in flight before either is counted
        for (int64_t i0 = k0 + (int64_t)tid * kHistRun; i0 < k1; i0 += 2 * kStep) {
            uint32_t a[kHistRun], b[kHistRun];
            const int ca = (int)min((int64_t)kHistRun, k1 - i0);
            const int cb = (int)max((int64_t)0, min((int64_t)kHistRun, k1 - i0 - kStep));
            if constexpr (FROM_F) {
                load_float_keys16(f, i0, ca, a, nan);
                if (cb > 0) load_float_keys16(f, i0 + kStep, cb, b, nan);
            } else {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    uint32_t(&k)[kHistRun] = h ? b : a;
                    const int c = h ? cb : ca;
                    const int64_t j0 = i0 + h * kStep;
                    if (c == kHistRun && vec) {
#pragma unroll
                        for (int q = 0; q < kHistRun / 4; ++q) {
                            const uint4 v = __ldcs(reinterpret_cast<const uint4*>(keys + j0) + q);
                            k[4 * q] = v.x;
                            k[4 * q + 1] = v.y;
                            k[4 * q + 2] = v.z;
                            k[4 * q + 3] = v.w;
                        }
                    } else {
#pragma unroll
                        for (int j = 0; j < kHistRun; ++j) k[j] = j < c ? keys[j0 + j] : 0u;
                    }
                }
            }
            count_runs_at(a, ca, SHIFT, wh);
            if (cb > 0) count_runs_at(b, cb, SHIFT, wh);
        }
        __syncthreads();
        uint32_t c = 0;
#pragma unroll
        for (int w = 0; w < kW; ++w) c += sh[w * kB + tid];
        cnt[(size_t)tid * kOrderMaxSuper + s] = c;
        mine += c;
        __syncthreads();
    }
    if (nan) record_error(status, MSC_ERR_NAN);
    if (mine) atomicAdd(&total[tid], mine);
}

// Scan: block d takes digit d.  Its super-tiles' counts become exclusive
// output positions starting at the digit's global start (the sum of the
// totals of the smaller digits); warp w scans the w-th eighth of the row.
__global__ void __launch_bounds__(kT) k_ord_scan(uint32_t* __restrict__ cnt, const uint32_t* __restrict__ total,
                                                 int supers) {
    __shared__ uint32_t s_w[kW];
    __shared__ uint32_t s_g;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int d = blockIdx.x;
    if (warp == 0) {
        uint32_t g = 0;
        for (int j = lane; j < d; j += 32) g += total[j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) g += __shfl_xor_sync(0xffffffffu, g, o);
        if (lane == 0) s_g = g;
    }
    uint32_t* row = cnt + (size_t)d * kOrderMaxSuper;
    constexpr int kPer = kOrderMaxSuper / kW / 32;  // entries per lane
    const int per_warp = (supers + kW - 1) / kW;
    const int b0 = warp * per_warp;
    uint32_t x[kPer], wsum = 0;
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
        const int i = j * 32 + lane;
        const int b = b0 + i;
        x[j] = (i < per_warp && b < supers) ? row[b] : 0u;
        wsum += x[j];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) wsum += __shfl_xor_sync(0xffffffffu, wsum, o);
    if (lane == 0) s_w[warp] = wsum;
    __syncthreads();
    uint32_t run = s_g;
    for (int w = 0; w < warp; ++w) run += s_w[w];
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
        if (j * 32 >= per_warp) break;
        uint32_t incl = x[j];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        const int i = j * 32 + lane;
        const int b = b0 + i;
        if (i < per_warp && b < supers) row[b] = run + incl - x[j];
        run += __shfl_sync(0xffffffffu, incl, 31);
    }
}

struct DownArgs {
    const float* f;            // pass 0: the field (keys made from it, ids implicit)
    const uint32_t* keys_in;   // other passes
    const int32_t* vals_in;
    uint32_t* keys_out;
    int32_t* vals_out;         // BUCKET: the ids of the filed pairs
    uint32_t* pair_pos;        // BUCKET: the positions of the filed pairs
    uint32_t* bucket_fill;     // BUCKET: slots taken per id bucket (stride kOrderFillStride)
    int bucket_shift;          // BUCKET: log2 of the ids per bucket
    Range r;
    const uint32_t* base;      // [256][kOrderMaxSuper] first output position per digit and super-tile
    const uint32_t* total;     // [256] keys per digit in this pass
    int use_tma;               // the inputs are 16-byte aligned: full tiles come by bulk copy
    int32_t* status;
};

// Shared memory of k_ord_down: two tile buffers of (key, value) words,
// warp histograms (16-bit; after the count, each warp's tile-local start),
// per-digit words, scan scratch, bucket words, two mbarriers.
constexpr size_t kBufWords = 2 * kTile;
constexpr size_t kDownSmem = 2 * kBufWords * 4 + kW * kB * 2 + 2 * kB * 4 + 32 * 4 + 2 * kB * 4 + 2 * 8;

// Lanes of the warp holding the same digit as this lane: one match
// instruction, whose cost grows with the number of distinct digits in the
// warp, or eight ballots, whose cost does not (digit_peers in radix.cuh).

template <bool FROM_F, bool BUCKET, int SHIFT>
__global__ void __launch_bounds__(kT, MSC_ORD_MIN_BLOCKS) k_ord_down(const DownArgs a) {
    extern __shared__ __align__(128) uint8_t smem[];
    uint32_t* buf = reinterpret_cast<uint32_t*>(smem);                     // [2][kTile words | kTile words]
    uint16_t* s_wh = reinterpret_cast<uint16_t*>(buf + 2 * kBufWords);     // [kW][kB]
    uint32_t* s_run = reinterpret_cast<uint32_t*>(s_wh + kW * kB);         // [kB] next output position
    uint32_t* s_delta = s_run + kB;                                        // [kB] output pos - staged pos
    uint32_t* s_misc = s_delta + kB;                                       // [32] scan scratch
    uint32_t* s_bcnt = s_misc + 32;                                        // [kB] BUCKET
    uint32_t* s_bbase = s_bcnt + kB;                                       // [kB] BUCKET
    uint64_t* mbar = reinterpret_cast<uint64_t*>(s_bbase + kB);            // [2]

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const Range r = a.r;
    if ((int)blockIdx.x >= r.supers) return;  // block-uniform
    // few populated digits in this pass (a float field's top byte): rank
    // with match, which is then cheaper than eight ballots (measured: 0.74
    // against 0.92 ms for the top byte of a 512^3 field)
    const bool use_match = __syncthreads_count(a.total[tid] != 0u) <= MSC_ORD_MATCH_MAX;
    const int64_t G = gridDim.x;
    // the tiles of this block in processing order: super-tiles
    // blockIdx.x, blockIdx.x + G, ..., each from its first tile to its last
    auto next_tile = [&](int64_t t) -> int64_t {
        if ((t + 1) % r.per_super != 0 && t + 1 < r.tiles) return t + 1;
        const int64_t s = t / r.per_super + G;
        return s < r.supers ? s * r.per_super : -1;
    };
    for (int i = tid; i < kW * kB / 2; i += kT) reinterpret_cast<uint32_t*>(s_wh)[i] = 0u;
    if (tid == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();

    const uint32_t* src_k = FROM_F ? reinterpret_cast<const uint32_t*>(a.f) : a.keys_in;
    // full, aligned tiles come by bulk copy; the ragged last tile by plain loads
    auto by_tma = [&](int64_t t) { return a.use_tma && (t + 1) * kTile <= r.n; };
    auto issue = [&](int64_t t, int slot) {  // one thread
        if (t < 0 || !by_tma(t)) return;
        uint32_t* dst = buf + slot * kBufWords;
        mbar_expect_tx(&mbar[slot], FROM_F ? kTile * 4 : kTile * 8);
        bulk_load(dst, src_k + t * kTile, kTile * 4, &mbar[slot]);
        if constexpr (!FROM_F) bulk_load(dst + kTile, a.vals_in + t * kTile, kTile * 4, &mbar[slot]);
    };
    int64_t t = (int64_t)blockIdx.x * r.per_super;
    if (tid == 0) issue(t, 0);

    const int wb = warp * (kI * 32) + lane;  // tile-local index of this thread's key k: wb + 32 k
    const uint32_t lt = lanemask_lt();
    uint16_t* wh = s_wh + warp * kB;
    for (int it = 0; t >= 0; ++it) {
        const int slot = it & 1;
        const int64_t tn = next_tile(t);
        // input: keys (or the field's words) in bk, values in bv; the keys are
        // staged into bv and the values into bk once each half has been read
        uint32_t* bk = buf + slot * kBufWords;
        uint32_t* bv = bk + kTile;
        if (tid == 0) issue(tn, slot ^ 1);
        // a super-tile starts: its output positions per digit (word tid is
        // read and written by thread tid only)
        if (t % r.per_super == 0) s_run[tid] = a.base[(size_t)tid * kOrderMaxSuper + t / r.per_super];
        const int cnt = (int)min((int64_t)kTile, r.n - t * kTile);
        const int64_t tb = t * kTile;
        if (by_tma(t)) {
            const bool ok = mbar_wait(&mbar[slot], (uint32_t)(it >> 1) & 1u, kWaitLimit);
            if (__syncthreads_or(!ok)) {
                // a copy never landed: report, let the prefetch in flight finish, stop
                if (tid == 0) {
                    record_error(a.status, MSC_ERR_INTERNAL);
                    if (tn >= 0 && by_tma(tn)) mbar_wait(&mbar[slot ^ 1], (uint32_t)((it + 1) >> 1) & 1u, kWaitLimit);
                }
                return;
            }
        } else {
            for (int i = tid; i < cnt; i += kT) {
                bk[i] = src_k[tb + i];
                if constexpr (!FROM_F) bv[i] = (uint32_t)a.vals_in[tb + i];
            }
            __syncthreads();
        }
        auto key_at = [&](int li) -> uint32_t {
            const uint32_t w = bk[li];
            return FROM_F ? float_key(__uint_as_float(w)) : w;
        };
        // stable rank among the warp's equal digits: earlier keys of the warp
        // (its 16-bit counter) + lower lanes of this step
        uint32_t rk[kI / 2];
        uint32_t dg[kI / 4];  // the digits of the thread's keys, four to a word
        // FULL: every key of the tile is valid (all but a ragged last tile)
        auto rank_tile = [&](auto match_tag, auto full_tag) {
            constexpr bool MATCH = decltype(match_tag)::value;
            constexpr bool FULL = decltype(full_tag)::value;
#pragma unroll
            for (int k = 0; k < kI; ++k) {
                const int li = wb + 32 * k;
                const bool valid = FULL || li < cnt;
                const uint32_t d = valid ? digit_of<SHIFT>(key_at(li)) : 0u;
                dg[k / 4] = (k & 3) ? (dg[k / 4] | d << (8 * (k & 3))) : d;
                uint32_t peers;
                if constexpr (MATCH) peers = __match_any_sync(0xffffffffu, valid ? d : 0x100u | lane);
                else if constexpr (FULL) peers = digit_peers_all(d);
                else peers = digit_peers(d, valid);
                const uint32_t lower = __popc(peers & lt);
                const uint32_t before = wh[d];
                if (valid && lower == 0) wh[d] = (uint16_t)(before + __popc(peers));
                const uint32_t rank = before + lower;
                rk[k / 2] = (k & 1) ? (rk[k / 2] | rank << 16) : rank;
                __syncwarp();
            }
        };
        if (cnt == kTile) {
            if (use_match) rank_tile(std::true_type{}, std::true_type{});
            else rank_tile(std::false_type{}, std::true_type{});
        } else {
            if (use_match) rank_tile(std::true_type{}, std::false_type{});
            else rank_tile(std::false_type{}, std::false_type{});
        }
        if constexpr (BUCKET) s_bcnt[tid] = 0u;
        __syncthreads();
        {   // digit tid: warp counts -> tile-local start of each warp's run of
            // the digit (16-bit: at most kTile); output start of the tile's run
            uint32_t pre[kW], run = 0;
#pragma unroll
            for (int w = 0; w < kW; ++w) {
                pre[w] = run;
                run += s_wh[w * kB + tid];
            }
            const uint32_t excl = block_scan_256(run, s_misc) - run;
#pragma unroll
            for (int w = 0; w < kW; ++w) s_wh[w * kB + tid] = (uint16_t)(excl + pre[w]);
            const uint32_t g = s_run[tid];
            s_delta[tid] = g - excl;
            s_run[tid] = g + run;
        }
        __syncthreads();
        if constexpr (!BUCKET) {
            // values into registers first (the field pass makes them from the
            // index), so that bv is free for the staged keys
            uint32_t val[kI];
            if constexpr (!FROM_F) {
#pragma unroll
                for (int k = 0; k < kI; ++k) val[k] = bv[wb + 32 * k];
                __syncthreads();
            }
            // each key to its tile-local sorted position; rk keeps the position
#pragma unroll
            for (int k = 0; k < kI; ++k) {
                const int li = wb + 32 * k;
                uint32_t lpos = 0;
                if (li < cnt) {
                    const uint32_t kk = key_at(li);
                    const uint32_t d = (dg[k / 4] >> (8 * (k & 3))) & 255u;
                    lpos = wh[d] + ((rk[k / 2] >> (16 * (k & 1))) & 0xffffu);
                    MSC_GUARD(lpos < (uint32_t)kTile, a.status, -141) bv[lpos] = kk;
                }
                rk[k / 2] = (k & 1) ? ((rk[k / 2] & 0xffffu) | lpos << 16) : ((rk[k / 2] & 0xffff0000u) | lpos);
            }
            __syncwarp();
            for (int j = lane; j < kB / 2; j += 32) reinterpret_cast<uint32_t*>(wh)[j] = 0u;
            __syncthreads();  // every key read: bk is free
#pragma unroll
            for (int k = 0; k < kI; ++k) {
                const int li = wb + 32 * k;
                if (li < cnt) {
                    const uint32_t lpos = (rk[k / 2] >> (16 * (k & 1))) & 0xffffu;
                    MSC_GUARD(lpos < (uint32_t)kTile, a.status, -141) bk[lpos] = FROM_F ? (uint32_t)(tb + li) : val[k];
                }
            }
            __syncthreads();
            // consecutive staged keys of one digit go to consecutive positions
#pragma unroll 4
            for (int k = 0; k < kI; ++k) {
                const int i = k * kT + tid;
                if (i < cnt) {
                    const uint32_t kk = bv[i];
                    const uint32_t pos = s_delta[digit_of<SHIFT>(kk)] + (uint32_t)i;
                    MSC_GUARD(pos < (uint64_t)r.n, a.status, -142) {
                        a.keys_out[pos] = kk;
                        a.vals_out[pos] = (int32_t)bk[i];
                    }
                }
            }
        } else {
            // final positions straight from the ranks; (id, position) pairs
            // regrouped by id bucket, each bucket's run written with
            // consecutive lanes on consecutive slots
            uint32_t ppos[kI], prank[kI / 2];
#pragma unroll
            for (int k = 0; k < kI; ++k) {
                const int li = wb + 32 * k;
                const uint32_t d = li < cnt ? (dg[k / 4] >> (8 * (k & 3))) & 255u : 0u;
                ppos[k] = s_delta[d] + wh[d] + ((rk[k / 2] >> (16 * (k & 1))) & 0xffffu);
            }
            __syncwarp();
            for (int j = lane; j < kB / 2; j += 32) reinterpret_cast<uint32_t*>(wh)[j] = 0u;
            uint32_t id[kI];
#pragma unroll
            for (int k = 0; k < kI; ++k) {
                if (k % 2 == 0) prank[k / 2] = 0u;
                const int li = wb + 32 * k;
                id[k] = bv[li];
                if (li < cnt) {
                    const uint32_t b = id[k] >> a.bucket_shift;
                    MSC_GUARD(b < (uint32_t)kB, a.status, -143)
                    prank[k / 2] |= atomicAdd(&s_bcnt[b], 1u) << (16 * (k & 1));
                }
            }
            __syncthreads();
            {
                const uint32_t c = s_bcnt[tid];
                const uint32_t start = block_scan_256(c, s_misc + 8) - c;
                s_bbase[tid] = c ? ((uint32_t)tid << a.bucket_shift) + atomicAdd(&a.bucket_fill[tid * kOrderFillStride], c)
                                 : 0u;
                s_bcnt[tid] = start;
            }
            __syncthreads();
#pragma unroll
            for (int k = 0; k < kI; ++k) {
                if (wb + 32 * k < cnt) {
                    const uint32_t j = s_bcnt[id[k] >> a.bucket_shift] + ((prank[k / 2] >> (16 * (k & 1))) & 0xffffu);
                    MSC_GUARD(j < (uint32_t)kTile, a.status, -144) {
                        bk[j] = ppos[k];
                        bv[j] = id[k];
                    }
                }
            }
            __syncthreads();
            for (int i = tid; i < cnt; i += kT) {
                const uint32_t v = bv[i];
                const uint32_t b = v >> a.bucket_shift;
                const uint32_t slot_ = s_bbase[b] + ((uint32_t)i - s_bcnt[b]);
                const uint32_t pos = bk[i];
                MSC_GUARD(slot_ < (uint64_t)r.n && pos < (uint64_t)r.n, a.status, -145) {
                    a.vals_out[slot_] = (int32_t)v;
                    a.pair_pos[slot_] = pos;
                }
            }
        }
        // this buffer is refilled by a bulk copy (async proxy) two tiles on
        fence_proxy_async_smem();
        __syncthreads();
        t = tn;
    }
}

template <bool FROM_F, bool BUCKET, int SHIFT>
int configure_down() {
    static int configured_dev = -1;  // the attribute is set once per device
    if (configured_dev != current_device().id) {
        MSC_TRY(cudaFuncSetAttribute(k_ord_down<FROM_F, BUCKET, SHIFT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kDownSmem));
        configured_dev = current_device().id;
    }
    return MSC_OK;
}

template <bool FROM_F, bool BUCKET, int SHIFT>
int launch_down(const DownArgs& a, int blocks, cudaStream_t s, const char* label) {
    const int rc = configure_down<FROM_F, BUCKET, SHIFT>();
    if (rc) return rc;
    {
        TraceScope ts_(label, s);
        k_ord_down<FROM_F, BUCKET, SHIFT><<<blocks, kT, kDownSmem, s>>>(a);
    }
    MSC_LAUNCHED();
    return MSC_OK;
}

template <bool FROM_F, int SHIFT>
int launch_up(const float* f, const uint32_t* keys, const Range& rg, int blocks, uint32_t* cnt, uint32_t* total,
              int32_t* status, cudaStream_t s) {
    {
        TraceScope ts_("order.up", s);
        k_ord_up<FROM_F, SHIFT><<<blocks, kT, 0, s>>>(f, keys, rg, cnt, total, status);
    }
    MSC_LAUNCHED();
    {
        TraceScope ts_("order.scan", s);
        k_ord_scan<<<kB, kT, 0, s>>>(cnt, total, rg.supers);
    }
    MSC_LAUNCHED();
    return MSC_OK;
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15) == 0; }

}  // namespace

int run_order(const float* f, int64_t n, int32_t* order, uint32_t* key_a, int32_t* id_a, uint32_t* key_b,
              int32_t* id_b, const SortScratch& sc, int32_t* status, cudaStream_t s) {
    if (n <= 0) return MSC_OK;
    Range rg;
    rg.n = n;
    rg.tiles = ceil_div(n, kTile);
    rg.per_super = ceil_div(rg.tiles, kOrderMaxSuper);
    rg.supers = (int)ceil_div(rg.tiles, rg.per_super);
    const int sms = current_device().sms;
    int occ = 0;
    {
        int rr = configure_down<false, false, 8>();
        if (rr) return rr;
        MSC_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_ord_down<false, false, 8>, kT, kDownSmem));
    }
    const int down_blocks = (int)std::min<int64_t>(rg.supers, (int64_t)sms * std::max(occ, 1));
    const int up_blocks = (int)std::min<int64_t>(rg.supers, (int64_t)sms * 4);
    uint32_t* cnt = sc.ord_cnt;
    uint32_t* totals = sc.ord_cnt + (size_t)kB * kOrderMaxSuper;  // [4][256]
    uint32_t* fill = totals + 4 * kB;
    MSC_TRY(cudaMemsetAsync(totals, 0, (4 * kB + kOrderMaxBuckets * kOrderFillStride) * sizeof(uint32_t), s));

    DownArgs a{};
    a.r = rg;
    a.base = cnt;
    a.status = status;
    a.f = f;
    int r;
    // pass 0: f -> (key_a, id_a)
    if ((r = launch_up<true, 0>(f, nullptr, rg, up_blocks, cnt, totals, status, s))) return r;
    a.keys_out = key_a;
    a.vals_out = id_a;
    a.total = totals;
    a.use_tma = aligned16(f);
    if ((r = launch_down<true, false, 0>(a, down_blocks, s, "order.down_first"))) return r;
    // pass 1: a -> b
    if ((r = launch_up<false, 8>(nullptr, key_a, rg, up_blocks, cnt, totals + kB, status, s))) return r;
    a.keys_in = key_a;
    a.vals_in = id_a;
    a.keys_out = key_b;
    a.vals_out = id_b;
    a.total = totals + kB;
    a.use_tma = aligned16(key_a) && aligned16(id_a);
    if ((r = launch_down<false, false, 8>(a, down_blocks, s, "order.down"))) return r;
    // pass 2: b -> a
    if ((r = launch_up<false, 16>(nullptr, key_b, rg, up_blocks, cnt, totals + 2 * kB, status, s))) return r;
    a.keys_in = key_b;
    a.vals_in = id_b;
    a.keys_out = key_a;
    a.vals_out = id_a;
    a.total = totals + 2 * kB;
    a.use_tma = aligned16(key_b) && aligned16(id_b);
    if ((r = launch_down<false, false, 16>(a, down_blocks, s, "order.down"))) return r;
    // pass 3: a -> (id, position) pairs filed by id bucket into (id_b, key_b)
    if ((r = launch_up<false, 24>(nullptr, key_a, rg, up_blocks, cnt, totals + 3 * kB, status, s))) return r;
    a.keys_in = key_a;
    a.vals_in = id_a;
    a.keys_out = nullptr;
    a.vals_out = id_b;
    a.pair_pos = key_b;
    a.bucket_fill = fill;
    a.bucket_shift = order_bucket_shift(n);
    a.total = totals + 3 * kB;
    a.use_tma = aligned16(key_a) && aligned16(id_a);
    if ((r = launch_down<false, true, 24>(a, down_blocks, s, "order.down_last"))) return r;
    // the inverse permutation; the last pass's inputs are free
    return order_invert(a.bucket_shift, id_b, key_b, id_a, key_a, sc.sub_fill, n, order, status, s);
}

}  // namespace msc
