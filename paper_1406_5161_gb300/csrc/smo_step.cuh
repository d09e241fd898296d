// Fused, persistent SMO step for sm_103a (kernel template; instantiated per
// row-pass arithmetic in smo_step_{binary,fp64,mixed}.cu).
//
// One cooperative launch runs many SMO iterations (Algorithm 1 / the loop of
// Algorithm 3 and, with shrinking, Algorithm 4) without returning to the
// host. Each CTA owns a contiguous segment of the samples (the sample
// partitioning of Algorithm 3, one segment per SM instead of one per MPI
// rank) and its active list pi_q (Algorithm 4). When the segment fits, its
// rows, f, alpha and index sets stay in shared memory for the whole launch
// ("resident" mode); otherwise they are streamed from global memory.
//
// One iteration:
//   1. every CTA loads x_up and x_low into a dense shared-memory target
//      buffer (the paper's MPI_Bcast of the two rows becomes two L2 reads);
//   2. every CTA computes K(up, low) from that buffer and the pair step of
//      Eq. (alphaup) with rho = -eta (Eq. rho) in FP64, identically, so no
//      exchange is needed;
//   3. the row pass: for each active sample i of the segment, the kernel
//      values K(up, i), K(low, i) (RBF via ||x||^2 + ||z||^2 - 2<x,z>), the
//      FP64 gradient update of Eq. (fup), on shrink iterations the rule of
//      Eq. (shrink), and the CTA's best I_up / I_low candidates;
//   4. a grid-wide exchange of the CTA candidates (the paper's
//      MPI_Allreduce "GlobalMinMax"): within a cluster through distributed
//      shared memory, between cluster leaders through global memory (slots
//      of epoch-tagged words, or release/acquire flags); every CTA reduces
//      the candidates in the same order and gets the same next pair
//      (Eq. bminmax, lowest index on ties);
//   5. on shrink iterations each CTA compacts its active list in place.
//
// All waits on other CTAs are bounded by a time limit; on expiry the kernel
// records an error and returns so the host can report SVM_ERR_TIMEOUT.
#pragma once

#include <climits>
#include <cstddef>
#include <type_traits>
#include <cooperative_groups.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "fp64_math.cuh"
#include "svm_internal.cuh"

namespace svmgb {
namespace smo {

constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;
constexpr int kMaxCluster = 16;    // largest thread-block cluster launched (non-portable size)
constexpr int kKcThread = 32;      // the kernel-row cache's directory keeper (lane 0 of warp 1)

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned ld_relaxed_u32(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

// named barrier 1 between the pair-step warp (arrives) and the row warps (wait)
__device__ __forceinline__ void step_bar_arrive(int n) { asm volatile("bar.arrive 1, %0;" ::"r"(n) : "memory"); }
__device__ __forceinline__ void step_bar_sync(int n) { asm volatile("bar.sync 1, %0;" ::"r"(n) : "memory"); }

__device__ __forceinline__ void st_release_u32(unsigned *p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Words of the several-cluster exchange: 32 bits of data in the low half of
// an 8-byte word whose high half is the epoch that wrote it. An aligned
// 8-byte access is single-copy atomic (each element of a .v2.b64 access is
// one), so a reader that finds its epoch in a word has that word's data: the
// data carry their own flag, with no fence behind the writer's stores and no
// second trip to L2 for the data after the flag.
__device__ __forceinline__ void st_tagged2(ulonglong2 *p, uint32_t d0, uint32_t d1, uint32_t ep)
{
    const unsigned long long w0 = ((unsigned long long)ep << 32) | d0, w1 = ((unsigned long long)ep << 32) | d1;
    asm volatile("st.relaxed.gpu.global.v2.b64 [%0], {%1, %2};" ::"l"(p), "l"(w0), "l"(w1) : "memory");
}
__device__ __forceinline__ ulonglong2 ld_tagged2(const ulonglong2 *p)
{
    ulonglong2 v;
    asm volatile("ld.relaxed.gpu.global.v2.b64 {%0, %1}, [%2];" : "=l"(v.x), "=l"(v.y) : "l"(p) : "memory");
    return v;
}

// Waits (acquire) until a leader's release flag reaches the given epoch;
// gives up after timeout_ns of %globaltimer, or at once when another CTA has
// flagged an error, and then flags the error itself.
static __device__ __noinline__ void wait_released(const unsigned *flag, unsigned need, long long timeout_ns, int *err)
{
    uint64_t t0 = 0;
    int spins = 0;
    while (ld_acquire_u32(flag) < need) {
        if (++spins >= 64) {
            spins = 0;
            if (*(volatile int *)err) return;
            uint64_t t;
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
            if (t0 == 0) t0 = t;
            else if (t - t0 > (uint64_t)timeout_ns) { atomicExch(err, 1); return; }
        }
    }
}

// named barrier 2 among the row warps only (warps 1..; the pair-step warp
// does not take part)
__device__ __forceinline__ void rows_bar_sync() { asm volatile("bar.sync 2, %0;" ::"r"(kThreads - 32) : "memory"); }

// D += A B on the tensor cores: A 16x16 BF16 (rows), B 16x8 BF16 (targets),
// D 16x8 FP32 (m16n8k16, register fragments)
__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                               uint32_t b0, uint32_t b1)
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
                 "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// distributed shared memory and mbarriers (32-bit shared-window addresses)
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint32_t cluster_addr(uint32_t a, int rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}
__device__ __forceinline__ void st_cluster_v4(uint32_t a, uint4 v)
{
    asm volatile("st.shared::cluster.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(a), "r"(v.x), "r"(v.y), "r"(v.z),
                 "r"(v.w)
                 : "memory");
}
// asynchronous store into a CTA of the cluster that counts its bytes on that
// CTA's mbarrier (no fence on the sending side)
__device__ __forceinline__ void st_async_v4(uint32_t a, uint4 v, uint32_t remote_bar)
{
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.b32 [%0], {%1, %2, %3, %4}, [%5];" ::"r"(a),
                 "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w), "r"(remote_bar)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_init(uint32_t bar, int count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t remote_bar)
{
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(remote_bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait_cluster(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok)
                 : "r"(bar), "r"(parity)
                 : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits for the phase of the given parity of a CTA-local mbarrier, giving up
// after timeout_ns of %globaltimer, or at once when another CTA has flagged
// an error; returns 1 when it gave up (the caller records the error and
// leaves its loop, so that no wait of the library can outlast its limit).
__device__ __forceinline__ int mbar_wait_bounded(uint32_t bar, uint32_t parity, int64_t timeout_ns, const int *err)
{
    int spins = 0;
    uint64_t t0 = 0;
    while (!mbar_try_wait_cluster(bar, parity)) {
        if (++spins >= 64) {
            spins = 0;
            const uint64_t now = global_ns();
            if (t0 == 0) t0 = now;
            else if (now - t0 > (uint64_t)timeout_ns) return 1;
            if (*(volatile const int *)err) return 1;
        }
    }
    return 0;
}

// status byte: bits 0-2 = index set (Eq. setinfo), bit 7 = label is +1
__device__ __forceinline__ uint8_t set_bits(uint8_t b) { return b & 7; }
__device__ __forceinline__ int8_t y_of(uint8_t b) { return (b & 0x80) ? 1 : -1; }
// One side (I_up or I_low) of a candidate: the sample and what the pair
// step needs about it, so that no CTA has to read another CTA's data.
struct Side {
    double f;       // gradient value
    double a;       // alpha
    double nrm;     // ||x||^2 (unused on binary input)
    int64_t p0;     // global CSR start of the row
    int32_t i;      // global sample index (INT_MAX when empty)
    int32_t len;    // CSR length of the row
    int32_t y;
    int32_t owner;  // cluster of the CTA whose segment holds the row
    uint32_t m[8];  // bit-mask modes: the row's bits (unused words zero)
};

struct __align__(16) CandFull {
    Side up, low;
    int32_t count;
    int32_t pad[3];
};
static_assert(sizeof(CandFull) % 16 == 0, "candidate slots are read with vector loads");
// the leader exchange reads a side's first 48 bytes as three 16-byte words
static_assert(offsetof(Side, f) == 0 && offsetof(Side, i) == 32 && offsetof(Side, m) == 48 &&
              sizeof(Side) % 16 == 0 && offsetof(CandFull, low) == sizeof(Side), "Side layout");
// global exchange slots: each candidate and each flag on lines of its own
constexpr size_t kCandStride = 256;
static_assert(sizeof(CandFull) <= kCandStride, "candidate slot too small");
// a leader's tagged slot: the first 48 bytes of both winning sides and the
// cluster's active count, 25 data words in 13 pairs
constexpr int kTagPairs = 13;
static_assert(kTagPairs * 16 <= (int)kCandStride, "tagged slot too small");

// Result of a step's exchange, written into every CTA of a cluster.
struct __align__(16) ResultArea {   // (sizeof a multiple of 16)
    Side up, low;
    long long total;   // active-set size over all segments
    int flag;          // a wait timed out
    int gap_open;      // b_low - b_up > the launch's threshold (Eq. kktterm): step on
};
// the several-cluster exchange writes a result as 16-byte words: the first
// 48 bytes of each side and (total, flag, gap_open)
static_assert(offsetof(ResultArea, low) == 80 && offsetof(ResultArea, total) == 160 &&
              offsetof(ResultArea, flag) == 168 && offsetof(ResultArea, gap_open) == 172, "ResultArea layout");

// FP64 compares and selects are long-latency on sm_103a; comparisons here
// use an order-preserving integer image of the double instead:
// dkey(a) < dkey(b) exactly when a < b (finite values, -0 taken as +0).
__device__ __forceinline__ unsigned long long dkey(double f)
{
    unsigned long long b = (unsigned long long)__double_as_longlong(f);
    if ((b << 1) == 0) b = 0;
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ bool dless(double a, double b) { return dkey(a) < dkey(b); }
// max(v, 0) of a squared distance, on the sign bit (no FP64 instruction)
__device__ __forceinline__ double dpos(double v) { return __double_as_longlong(v) < 0 ? 0.0 : v; }
__device__ __forceinline__ double neg_if(double v, bool neg)
{
    return neg ? __longlong_as_double(__double_as_longlong(v) ^ (long long)0x8000000000000000ull) : v;
}
// index set of a snapped alpha (exactly 0, exactly C, or in between)
__device__ __forceinline__ uint8_t status_of(bool ypos, double a, double C)
{
    const long long b = __double_as_longlong(a);
    uint8_t set;
    if (b == 0) set = ypos ? ST_I1 : ST_I4;
    else if (b == __double_as_longlong(C)) set = ypos ? ST_I3 : ST_I2;
    else set = ST_I0;
    return (uint8_t)(set | (ypos ? 0x80 : 0));
}

// Selection keys: the I_up side minimises f, the I_low side maximises it;
// both become a minimum over (key, index), so ties go to the lowest index.
__device__ __forceinline__ unsigned long long key_up(double f) { return dkey(f); }
__device__ __forceinline__ unsigned long long key_low(double f) { return ~dkey(f); }
constexpr unsigned long long kNoKey = ~0ull;

__device__ __forceinline__ bool ki_less(unsigned long long k, int i, unsigned long long bk, int bi)
{
    return k < bk || (k == bk && i < bi);
}

// Warp minimum of (key, index) in lexicographic order; every lane ends with
// the winner. Three 32-bit warp reductions (high key word, low key word
// among the lanes that hold the least high word, index among the lanes that
// hold the least key); indices are non-negative, INT_MAX marks no candidate.
__device__ __forceinline__ void warp_min_ki(unsigned long long &k, int &i)
{
    const unsigned hi = (unsigned)(k >> 32), lo = (unsigned)k;
    const unsigned mhi = __reduce_min_sync(0xffffffffu, hi);
    const unsigned mlo = __reduce_min_sync(0xffffffffu, hi == mhi ? lo : 0xffffffffu);
    const unsigned mi = __reduce_min_sync(0xffffffffu, (hi == mhi && lo == mlo) ? (unsigned)i : 0xffffffffu);
    k = ((unsigned long long)mhi << 32) | mlo;
    i = (int)mi;
}

__device__ __forceinline__ void side_empty(Side &s, bool up)
{
    s.f = up ? __longlong_as_double(0x7ff0000000000000ll) : __longlong_as_double(0xfff0000000000000ll);
    s.a = 0.0;
    s.nrm = 0.0;
    s.p0 = 0;
    s.i = INT_MAX;
    s.len = 0;
    s.y = 0;
    s.owner = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) s.m[w] = 0;
}

// Word-wise copies of a candidate side (few live registers; generic
// destinations may be another CTA's shared memory).
__device__ __forceinline__ void copy_side(Side *dst, const Side *src)
{
    const unsigned long long *s = reinterpret_cast<const unsigned long long *>(src);
    unsigned long long *d = reinterpret_cast<unsigned long long *>(dst);
#pragma unroll
    for (int w = 0; w < (int)(sizeof(Side) / 8); ++w) d[w] = s[w];
}
__device__ __forceinline__ void copy_side_ldcg(Side *dst, const Side *src)   // src in global memory
{
    const unsigned long long *s = reinterpret_cast<const unsigned long long *>(src);
    unsigned long long *d = reinterpret_cast<unsigned long long *>(dst);
#pragma unroll
    for (int w = 0; w < (int)(sizeof(Side) / 8); ++w) d[w] = __ldcg(s + w);
}
__device__ __forceinline__ void copy_result(ResultArea *dst, const ResultArea *src)
{
    const uint4 *s = reinterpret_cast<const uint4 *>(src);
    uint4 *d = reinterpret_cast<uint4 *>(dst);
#pragma unroll
    for (int w = 0; w < (int)(sizeof(ResultArea) / 16); ++w) d[w] = s[w];
}
__device__ __forceinline__ uint4 shfl_u4(uint4 v, int src)
{
    return make_uint4(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src),
                      __shfl_sync(0xffffffffu, v.z, src), __shfl_sync(0xffffffffu, v.w, src));
}
// (key, index) of the I_up and I_low sides of a candidate
__device__ __forceinline__ void cand_keys(const CandFull &c, unsigned long long &k1, int &i1,
                                          unsigned long long &k2, int &i2, long long &cnt)
{
    i1 = c.up.i;
    i2 = c.low.i;
    k1 = i1 == INT_MAX ? kNoKey : key_up(c.up.f);
    k2 = i2 == INT_MAX ? kNoKey : key_low(c.low.f);
    cnt = c.count;
}

// Block-wide exclusive scan of 0/1 flags; returns the prefix, total in *tot.
__device__ __forceinline__ int block_scan_flag(bool flag, int *warp_sums, int *tot)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned m = __ballot_sync(0xffffffffu, flag);
    int pre = __popc(m & ((1u << lane) - 1u));
    if (lane == 0) warp_sums[w] = __popc(m);
    __syncthreads();
    if (w == 0) {
        int v = lane < kWarps ? warp_sums[lane] : 0;
        int incl = v;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            int o = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += o;
        }
        if (lane < kWarps) warp_sums[lane] = incl - v;
        if (lane == 31) *tot = incl;
    }
    __syncthreads();
    return pre + warp_sums[w];
}

template <int MODE>
struct RowMath;
template <>
struct RowMath<MODE_BINARY> {
    using Acc = int;
    using Tgt = unsigned short;  // byte 0: column of x_up set, byte 1: of x_low
    using Nrm = float;           // unused
};
template <>
struct RowMath<MODE_FP64> {
    using Acc = double;
    using Tgt = double2;         // .x value of x_up, .y value of x_low
    using Nrm = double;
};
template <>
struct RowMath<MODE_MIXED> {
    using Acc = float;
    using Tgt = float2;
    using Nrm = float;
};
template <>
struct RowMath<MODE_BITS4> {
    using Acc = int;
    using Tgt = unsigned char;   // unused: the targets are the masks in registers
    using Nrm = float;           // unused
};
template <>
struct RowMath<MODE_BITS8> : RowMath<MODE_BITS4> {};

struct Shared {
    Side wup[kWarps], wlow[kWarps];           // per-warp winners of the row pass
    unsigned long long wkup[kWarps], wklow[kWarps];
    int wiup[kWarps], wilow[kWarps];
    Side rup[8], rlow[8];                     // per-warp winners of the exchange
    unsigned long long rkup[8], rklow[8];
    int riup[8], rilow[8], rto[8];
    unsigned rrel[kWarps];                    // several clusters: least epoch seen released by every leader, per warp
    CandFull ccand[kMaxCluster];              // cluster leader: its CTAs' candidates
    CandFull xc[2][kMaxCluster];              // one cluster: every CTA's candidate, by epoch parity
    Side none[2];                             // empty I_up / I_low sides
    int kc_su, kc_sl, kc_hu, kc_hl;           // kernel-row cache: slots of x_up / x_low, hits
    double kc_kul;                            // FP64: K(up, low) from x_up's cached row (on a hit)
    unsigned long long xbar[2];               // one cluster: mbarriers of the two parities
    ResultArea res;                           // exchange result pushed by the leader
    long long rcount[8];
    int scan[kWarps];
    int scan_tot;
    double du, dl;        // y_up * delta alpha_up, y_low * delta alpha_low
    double au_new, al_new;
    unsigned char st_u, st_l;
    int flag_timeout;
};

template <int MODE>
__device__ __forceinline__ void tgt_clear(typename RowMath<MODE>::Tgt &t)
{
    if constexpr (MODE == MODE_BINARY || mode_bits(MODE)) t = 0;
    else if constexpr (MODE == MODE_FP64) t = make_double2(0.0, 0.0);
    else t = make_float2(0.f, 0.f);
}

// FP64 target entry, side 0 (x_up) or 1 (x_low): the value as a double, or,
// with exact inner products, (m, b + te_off) as two ints in the double's
// place (te_off = bias + t, so that a row entry's b - t plus it is the shift
// k = b_x + b_z + bias)
template <int SIDE>
__device__ __forceinline__ void xd_put(double2 &t, float v, bool xd, int tmin, int te_off)
{
    double w;
    if (xd) {
        const uint32_t u = __float_as_uint(v);
        w = __hiloint2double(xd_exp(u, tmin) + te_off, xd_mant(u));
    } else {
        w = (double)v;
    }
    if (SIDE == 0) t.x = w;
    else t.y = w;
}

// the exact partial sums of LPR consecutive lanes, added in every one of them
template <int LPR>
__device__ __forceinline__ void xd_lane_sum(XdAcc &a)
{
#pragma unroll
    for (int off = LPR / 2; off >= 1; off >>= 1) {
        XdAcc b;
        b.w0 = __shfl_xor_sync(0xffffffffu, a.w0, off);
        b.w1 = __shfl_xor_sync(0xffffffffu, a.w1, off);
        b.w2 = __shfl_xor_sync(0xffffffffu, a.w2, off);
        b.w3 = __shfl_xor_sync(0xffffffffu, a.w3, off);
        xd_add(a, b);
    }
}

// SOLO: the grid is one thread-block cluster (exchange through distributed
// shared memory only); a separate instantiation, so that the kernels for
// several clusters carry none of its code. WSS: i_low by the second-order
// gain (a second sweep and exchange per step), also its own instantiation.
template <int MODE, int LPR, bool RES, bool SOLO, bool WSS>
__global__ void __launch_bounds__(kThreads, 1) smo_persistent_kernel(SmoArgs A)
{
    using Tgt = typename RowMath<MODE>::Tgt;
    using Acc = typename RowMath<MODE>::Acc;
    using Nrm = typename RowMath<MODE>::Nrm;
    constexpr bool BITS = mode_bits(MODE);
    constexpr int W4 = mode_words(MODE) / 4;   // uint4 words of a bit-mask row
    extern __shared__ __align__(16) unsigned char dsm[];
    __shared__ Shared sh;
    // FP64 rows: 2^(-j/256) in Q63 for the fixed-point exp of the row pass
    __shared__ uint64_t expfx_s[MODE == MODE_FP64 ? kExpfxTabLen : 1];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int G = A.G, cta = blockIdx.x;
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    const int csize = (int)cluster.num_blocks();   // CTAs per cluster (1 without clusters)
    const int crank = (int)cluster.block_rank();
    const int cid = cta / csize;                   // cluster index = leader slot
    const int nlead = G / csize;
    // warps that poll the exchange slots; the warp after them releases the
    // leader's epochs and the rest record those of all leaders (FP64 cache)
    const int xwarps = (nlead + 31) / 32;
    // leaders' slots as tagged words when one warp polls them all; a flat
    // launch over more CTAs (every slot read by every CTA) and bit-mask rows
    // use a release flag per slot and read only what they need after it
    const bool tagged = !BITS && nlead <= 32;
    // the leaders' release flags for the FP64 kernel-row cache
    auto rel_flag = [&](int c) { return A.seq + ((size_t)2 * nlead + c) * kSeqStride; };
    const int d = A.d;
    // kernel-row cache: K(x_up, .) and K(x_low, .) of recent steps, per CTA
    // segment, in device memory (FP64 and mixed modes)
    constexpr bool KC_MODE = MODE == MODE_FP64 || MODE == MODE_MIXED;
    using KT = typename std::conditional<MODE == MODE_FP64, double, float>::type;
    const bool kc_on = KC_MODE && A.kc != nullptr;
    const SmoLayout L = smo_layout(MODE, d, A.ktab_len, A.maxnnz, RES ? 1 : 0, A.seg_rows_max,
                                   A.seg_nnz_max,
                                   kc_on ? smo_kdir_bytes(A.n, A.kc_slots, A.kc_direct) : 0);
    uint32_t *kdir = reinterpret_cast<uint32_t *>(dsm + L.kdir);
    Tgt *tbuf = reinterpret_cast<Tgt *>(dsm + L.tgt);            // [2][d]
    int *tcol = reinterpret_cast<int *>(dsm + L.tcol);           // [2 buf][2 side][maxnnz]
    double *ktab = reinterpret_cast<double *>(dsm + L.ktab);
    double *f_s = reinterpret_cast<double *>(dsm + L.f);
    double *a_s = reinterpret_cast<double *>(dsm + L.alpha);
    Nrm *nrm_s = reinterpret_cast<Nrm *>(dsm + L.nrm);
    int *rp_s = reinterpret_cast<int *>(dsm + L.rowptr);
    int *act_s = reinterpret_cast<int *>(dsm + L.act);
    uint8_t *st_s = reinterpret_cast<uint8_t *>(dsm + L.st);
    unsigned short *col_s = reinterpret_cast<unsigned short *>(dsm + L.col);
    float *val_s = reinterpret_cast<float *>(dsm + L.val);
    uint4 *bits_s = reinterpret_cast<uint4 *>(dsm + L.bits);
    uint32_t *dist_s = reinterpret_cast<uint32_t *>(dsm + L.dist);   // bit-mask rows on chip
    const uint4 *bits_g = reinterpret_cast<const uint4 *>(A.bits);
    const int maxnnz = A.maxnnz > 0 ? A.maxnnz : 1;

    const int64_t lo = seg_lo(A.n, G, cta);
    const int nseg = (int)(seg_lo(A.n, G, cta + 1) - lo);
    const int64_t base = A.indptr[lo];   // global CSR offset of the segment

    // FP64 mode with exact inner products (A.xd.on): a target entry holds, as
    // four ints, (m, b) of x_up's value and (m, b) of x_low's value at its
    // column (xd_mant, xd_exp); an absent value is m = 0, b = tmin
    const bool xd = MODE == MODE_FP64 && A.xd.on;
    const int xd_tmin = A.xd.tmin, xd_bias = A.xd.bias, xd_unit = A.xd.unit;
    // target entries hold b + te_off: a row entry's word adds its b - t
    const int xd_te = xd_bias + xd_tmin;
    Tgt tclear;
    tgt_clear<MODE>(tclear);
    if constexpr (MODE == MODE_FP64) {
        // an absent value: m = 0, b = t
        if (xd) tclear = make_double2(__hiloint2double(xd_tmin + xd_te, 0), __hiloint2double(xd_tmin + xd_te, 0));
    }
    // ---- set-up
    if constexpr (!BITS) {
        for (int c = tid; c < 2 * d; c += kThreads) tbuf[c] = tclear;
    }
    if constexpr (MODE == MODE_BINARY || BITS) {
        for (int c = tid; c < 3 * A.ktab_len; c += kThreads) ktab[c] = A.ktab[c];
    }
    if constexpr (MODE == MODE_FP64) {
        for (int c = tid; c < kExpfxTabLen; c += kThreads) expfx_s[c] = kExpfxTab[c];
    }
    const double *rtab = ktab + A.ktab_len;      // 1 / eta (0 when eta <= 1e-12)
    const double *etab = ktab + 2 * A.ktab_len;  // eta = 2 - 2 exp(-gamma k)
    int cnt = A.seg_cnt[cta];
    if constexpr (RES) {
        for (int r = tid; r < nseg; r += kThreads) {
            f_s[r] = A.f[lo + r];
            a_s[r] = A.alpha[lo + r];
            st_s[r] = A.status[lo + r];
            if constexpr (!BITS) rp_s[r] = (int)(A.indptr[lo + r] - base);
            if constexpr (MODE == MODE_FP64) nrm_s[r] = A.norm[lo + r];
            if constexpr (MODE == MODE_MIXED) nrm_s[r] = A.normf[lo + r];
        }
        if constexpr (BITS) {
            for (int q = tid; q < nseg * W4; q += kThreads) bits_s[q] = bits_g[(size_t)lo * W4 + q];
        } else {
            if (tid == 0) rp_s[nseg] = (int)(A.indptr[lo + nseg] - base);
            const int64_t segnnz = A.indptr[lo + nseg] - base;
            for (int64_t p = tid; p < segnnz; p += kThreads) {
                if constexpr (MODE == MODE_MIXED) {
                    // one word per entry: the column and the BF16 value
                    reinterpret_cast<uint32_t *>(val_s)[p] = A.ew[base + p];
                } else {
                    col_s[p] = (unsigned short)A.indices[base + p];
                    if constexpr (MODE == MODE_FP64) {
                        // exact inner products: the value's (m, b - t) word
                        const float v = A.values[base + p];
                        if (xd) reinterpret_cast<uint32_t *>(val_s)[p] = xd_word(__float_as_uint(v), xd_tmin);
                        else val_s[p] = v;
                    }
                }
            }
        }
        for (int k = tid; k < cnt; k += kThreads) act_s[k] = A.act[lo + k];
    }
    if (kc_on) {
        // empty directory: no valid rows (direct), no tags and zero stamps (4-way sets)
        if (A.kc_direct) {
            for (int w = tid; w < (int)((A.n + 31) / 32); w += kThreads) kdir[w] = 0;
        } else {
            for (int w = tid; w < A.kc_slots; w += kThreads) {
                kdir[w] = 0xffffffffu;
                kdir[A.kc_slots + w] = 0;
            }
        }
    }
    int64_t kc_hits = 0, kc_misses = 0;
    SmoCtrl C0 = *A.ctrl;
    int64_t iter = C0.iter, counter = C0.counter, row_visits = C0.row_visits;
    int64_t shrink_events = C0.shrink_events;
    long long total = C0.active;
    int64_t ph[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (tid == 0) sh.flag_timeout = 0;
    Side up, low;
    side_empty(up, true);
    side_empty(low, false);
    auto load_mask = [&](Side &sd) {
        if constexpr (BITS) {
#pragma unroll
            for (int q = 0; q < W4; ++q) {
                const uint4 v = bits_g[(size_t)sd.i * W4 + q];
                sd.m[4 * q] = v.x; sd.m[4 * q + 1] = v.y; sd.m[4 * q + 2] = v.z; sd.m[4 * q + 3] = v.w;
            }
        }
    };
    bool first = A.select_only != 0;
    if (!first) {
        up.f = C0.b_up; up.a = C0.a_up; up.i = C0.i_up;
        low.f = C0.b_low; low.a = C0.a_low; low.i = C0.i_low;
        if (up.i >= 0 && up.i < A.n) {
            up.p0 = A.indptr[up.i];
            up.len = (int)(A.indptr[up.i + 1] - up.p0);
            up.y = A.y[up.i];
            up.nrm = MODE == MODE_MIXED ? (double)A.normf[up.i] : (MODE == MODE_FP64 ? A.norm[up.i] : 0.0);
            load_mask(up);
        }
        if (low.i >= 0 && low.i < A.n) {
            low.p0 = A.indptr[low.i];
            low.len = (int)(A.indptr[low.i + 1] - low.p0);
            low.y = A.y[low.i];
            low.nrm = MODE == MODE_MIXED ? (double)A.normf[low.i] : (MODE == MODE_FP64 ? A.norm[low.i] : 0.0);
            load_mask(low);
        }
    }
    // one cluster over the whole grid: candidates go to every CTA as
    // asynchronous stores whose bytes each CTA counts on its own mbarrier
    // (one per epoch parity; the CTA's own arrival sets the expected bytes)
    constexpr bool solo = SOLO;
    if (tid == 0) {
        side_empty(sh.none[0], true);
        side_empty(sh.none[1], false);
    }
    if constexpr (SOLO) {
        if (nlead != 1) {   // launched over several clusters: refuse
            if (tid == 0) atomicExch(&A.ctrl->err, 1);
            return;
        }
        if (tid == 0) {
            mbar_init(smem_u32(&sh.xbar[0]), 1);
            mbar_init(smem_u32(&sh.xbar[1]), 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        __syncthreads();
        cluster.sync();
    } else {
        __syncthreads();
    }

    // ---- accessors (segment-local row r, global sample lo + r)
    auto ACT = [&](int k) -> int {
        if constexpr (RES) return act_s[k];
        else return A.act[lo + k];
    };
    auto SET_ACT = [&](int k, int v) {
        if constexpr (RES) act_s[k] = v;
        else A.act[lo + k] = v;
    };
    auto ROWP = [&](int r, int64_t &p0, int64_t &p1) {
        if constexpr (RES) { p0 = rp_s[r]; p1 = rp_s[r + 1]; }
        else { p0 = A.indptr[lo + r]; p1 = A.indptr[lo + r + 1]; }
    };
    // mixed rows on chip: one word per entry, the column in the low half and
    // the BF16 value's bits in the high half
    auto COL = [&](int64_t p) -> int {
        if constexpr (RES && MODE == MODE_MIXED) return (int)(reinterpret_cast<const uint32_t *>(val_s)[p] & 0xffffu);
        else if constexpr (RES) return (int)col_s[p];
        else return A.indices[p];
    };
    auto VAL = [&](int64_t p) -> float {
        if constexpr (RES && MODE == MODE_MIXED)
            return __uint_as_float(reinterpret_cast<const uint32_t *>(val_s)[p] & 0xffff0000u);
        else if constexpr (RES) return val_s[p];
        else if constexpr (MODE == MODE_FP64) return A.values[p];
        else return A.vmix[p];
    };
    // FP64 with exact inner products: entry p's column and (m, b - t) word
    // (on chip: the word is in place of the value; streamed: from the packed
    // 64-bit entries when there are some)
    auto XCW = [&](int64_t p, int &c, uint32_t &w) {
        if constexpr (RES) {
            c = (int)col_s[p];
            w = reinterpret_cast<const uint32_t *>(val_s)[p];
        } else {
            if (A.ew64) {
                const uint64_t e = A.ew64[p];
                c = (int)(e & 0xffffu);
                w = (uint32_t)(e >> 16);
            } else {
                c = A.indices[p];
                w = xd_word(__float_as_uint(A.values[p]), xd_tmin);
            }
        }
    };
    auto GETF = [&](int r) -> double {
        if constexpr (RES) return f_s[r];
        else return A.f[lo + r];
    };
    auto PUTF = [&](int r, double v) {
        if constexpr (RES) f_s[r] = v;
        else A.f[lo + r] = v;
    };
    auto GETST = [&](int r) -> uint8_t {
        if constexpr (RES) return st_s[r];
        else return A.status[lo + r];
    };
    auto PUTST = [&](int r, uint8_t v) {
        if constexpr (RES) st_s[r] = v;
        else A.status[lo + r] = v;
    };
    auto GETA = [&](int r) -> double {
        if constexpr (RES) return a_s[r];
        else return A.alpha[lo + r];
    };
    auto PUTA = [&](int r, double v) {
        if constexpr (RES) a_s[r] = v;
        else A.alpha[lo + r] = v;
    };
    auto NRM = [&](int r) -> double {
        if constexpr (MODE == MODE_BINARY || BITS) return 0.0;
        else if constexpr (RES) return (double)nrm_s[r];
        else if constexpr (MODE == MODE_FP64) return A.norm[lo + r];
        else return (double)A.normf[lo + r];
    };
    // mixed mode: the FP32 norm as it is stored (no round trip through the
    // FP64 pipe, whose conversions cost as much as its arithmetic here)
    auto NRMF = [&](int r) -> float {
        if constexpr (MODE != MODE_MIXED) return 0.f;
        else if constexpr (RES) return nrm_s[r];
        else return A.normf[lo + r];
    };

    const double C = A.C;
    const double snap = 1e-12 * C, c_snap = C - snap;
    const float gammaf = (float)A.gamma;
    unsigned epoch = 0;
    int kc_pf0 = -1, kc_pf1 = -1;   // directory keeper: cache slots filled in the previous step
    int exit_reason = 0;
    bool gap_open = first || dless(A.thr, low.f - up.f);   // stopping test of the pair in up / low
    int prev_valid = 0;              // buffer (1 - buf) holds the previous targets
    int prev_len_u = 0, prev_len_l = 0;
    // optional per-phase cycle counts of CTA 0 (one clock read per phase)
    const bool timed = A.phase_times && cta == 0;
    uint64_t tp = (timed && tid == 0) ? clock64() : 0;
    // with phase_times every CTA counts the cycles from step start to publish
    const bool busy_on = A.phase_times && A.cta_cycles;
    uint64_t cta_t0 = 0, busy = 0;
    // second-order selection: low is the gain winner, beta_low the first-order
    // b_low (Eq. bminmax) that the shrink rule and the stopping test read
    double beta_low = low.f;

    for (;;) {
        const int buf = (int)(iter & 1);
        Tgt *T = tbuf + (size_t)buf * d;
        int *tcu = tcol + (size_t)(buf * 2 + 0) * maxnnz;
        int *tcl = tcol + (size_t)(buf * 2 + 1) * maxnnz;
        bool shrink_now = false;
        const double bup_sel = up.f, blow_sel = WSS ? beta_low : low.f;   // values that chose this pair
        if (busy_on && tid == 0) cta_t0 = clock64();
        if (!first) {
            if (!gap_open) { exit_reason = 0; break; }
            if (iter >= A.iter_limit) { exit_reason = 1; break; }
            if (total < A.compact_below) { exit_reason = 2; break; }
            // ---- 0. kernel-row cache: this step's rows of x_up and x_low
            //         (the same decisions in every CTA; a row found here was
            //         stored by this CTA in an earlier step of this launch)
            // (by lane 0 of warp 1, which has no part in the target fill of
            // short rows, so that the FP64 K(up, low) it reads from the cache
            // arrives while the other threads fill the targets)
            if (kc_on && tid == kKcThread) {
                auto lookup = [&](int i, int &slot, int &hit) {
                    if (A.kc_direct) {
                        const uint32_t bit = 1u << (i & 31);
                        hit = (kdir[i >> 5] & bit) != 0;
                        kdir[i >> 5] |= bit;
                        slot = i;
                    } else {
                        const int nsets = A.kc_slots >> 2;
                        const int set = i % nsets;
                        uint32_t *tags = kdir + 4 * set, *stamps = kdir + A.kc_slots + 4 * set;
                        int way = -1;
#pragma unroll
                        for (int w = 0; w < 4; ++w)
                            if (tags[w] == (uint32_t)i) way = w;
                        hit = way >= 0;
                        if (!hit) {   // least recently used way
                            way = 0;
#pragma unroll
                            for (int w = 1; w < 4; ++w)
                                if (stamps[w] < stamps[way]) way = w;
                            tags[way] = (uint32_t)i;
                        }
                        stamps[way] = (uint32_t)(iter + 1);
                        slot = 4 * set + way;
                    }
                };
                int su_, hu_, sl_, hl_;
                lookup(up.i, su_, hu_);
                lookup(low.i, sl_, hl_);
                sh.kc_su = su_; sh.kc_hu = hu_;
                sh.kc_sl = sl_; sh.kc_hl = hl_;
                kc_hits += hu_ + hl_;
                kc_misses += 2 - hu_ - hl_;
                if constexpr (MODE == MODE_FP64) {
                    if (hu_) {
                        // the entry was written by the CTA that owns x_low's
                        // row. Several clusters: its leader's release of an
                        // epoch after the write, acquired by this CTA's spare
                        // warps during the last exchange (the least epoch
                        // they saw released by every leader is in sh.rrel)
                        // or here, makes it visible: the epoch just ended for
                        // a slot filled in the previous step, else the one
                        // before
                        if constexpr (!SOLO) {
                            const unsigned need = (su_ == kc_pf0 || su_ == kc_pf1) ? epoch : epoch - 1u;
                            unsigned seen = 0xffffffffu;
                            for (int w = xwarps + 1; w < kWarps; ++w) seen = min(seen, sh.rrel[w]);
                            if (seen < need)
                                wait_released(rel_flag(low.owner), need, A.timeout_ns, &A.ctrl->err);
                        }
                        sh.kc_kul = __ldcg(static_cast<const double *>(A.kc) + (size_t)su_ * A.kc_ld + low.i);
                    }
                    kc_pf0 = hu_ ? -1 : su_;
                    kc_pf1 = hl_ ? -1 : sl_;
                }
            }
            // ---- 1. targets: x_up into .x / byte 0, x_low into .y / byte 1
            //         (bit-mask modes: the masks came with the exchange); x_up
            //         by the first half of the threads and x_low by the
            //         second, so that the loads of both rows are in flight
            //         together (one round trip to L2, not two)
            if constexpr (!BITS) {
                constexpr int kHalf = kThreads / 2;
                if (tid < kHalf) {
                    for (int k = tid; k < up.len; k += kHalf) {
                        int c = A.indices[up.p0 + k];
                        tcu[k] = c;
                        if constexpr (MODE == MODE_BINARY) reinterpret_cast<unsigned char *>(T + c)[0] = 1;
                        else if constexpr (MODE == MODE_FP64) xd_put<0>(T[c], A.values[up.p0 + k], xd, xd_tmin, xd_te);
                        else T[c].x = A.vmix[up.p0 + k];
                    }
                } else {
                    for (int k = tid - kHalf; k < low.len; k += kHalf) {
                        int c = A.indices[low.p0 + k];
                        tcl[k] = c;
                        if constexpr (MODE == MODE_BINARY) reinterpret_cast<unsigned char *>(T + c)[1] = 1;
                        else if constexpr (MODE == MODE_FP64) xd_put<1>(T[c], A.values[low.p0 + k], xd, xd_tmin, xd_te);
                        else T[c].y = A.vmix[low.p0 + k];
                    }
                }
            }
            if (A.h > 0) {
                counter -= 1;
                shrink_now = counter <= 0;
            }
            row_visits += total;
            if constexpr (!BITS) __syncthreads();
            if (timed && tid == 0) { uint64_t t = clock64(); ph[0] += t - tp; tp = t; }
        }

        // ---- 2. the pair step (warp 0) runs while warps 1.. compute the
        //         row sums and kernel values; the f updates wait for it on a
        //         named barrier.
        unsigned long long bku = kNoKey, bkl = kNoKey;   // this thread's best keys
        int biu = INT_MAX, bil = INT_MAX;                // ... their sample indices
        int bru = 0, brl = 0;                            // ... and segment rows
        if (warp == 0) {
            if (!first) {
                Acc s = 0;
                bool kul_cached = false;   // FP64: K(up, low) read from the kernel-row cache
                double kul_c = 0.0;
                if constexpr (BITS) {
                    // ||x_up - x_low||^2 of binary rows
#pragma unroll
                    for (int w = 0; w < 4 * W4; ++w) s += __popc(up.m[w] ^ low.m[w]);
                } else if constexpr (MODE == MODE_FP64) {
                    // K(up, low) with the row pass's own arithmetic for the
                    // row of x_low against the x_up target (exact inner
                    // products; else its entries in order, split over LPR
                    // lanes as the row pass splits a row), so that it equals,
                    // bit for bit, the entry the kernel-row cache holds for
                    // it and the value the row pass computes; when x_up's row is in
                    // the cache that entry is read instead (written by the
                    // owner of x_low's segment in an earlier step of this
                    // launch, visible here through the exchanges since)
                    if (kc_on && sh.kc_hu) {
                        kul_c = sh.kc_kul;
                        kul_cached = true;
                    } else if (xd) {
                        // exact: the same value whatever the order or split,
                        // so all 32 lanes share the entries
                        const int4 *T4 = reinterpret_cast<const int4 *>(T);
                        XdAcc a = xd_zero();
                        for (int k = lane; k < low.len; k += 32) {
                            const int4 t = T4[tcl[k]];
                            xd_add(a, t.z, t.x, t.w + t.y - (xd_te + xd_tmin));
                        }
                        xd_lane_sum<32>(a);
                        s = xd_round(a, xd_unit);
                    } else {
                        if (lane < LPR) {
                            for (int k = lane; k < low.len; k += LPR) {
                                const Tgt t = T[tcl[k]];
                                s = fma(t.y, t.x, s);
                            }
                        }
#pragma unroll
                        for (int off = LPR / 2; off >= 1; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
                    }
                } else {
                    for (int k = lane; k < low.len; k += 32) {
                        const Tgt t = T[tcl[k]];
                        if constexpr (MODE == MODE_BINARY) s += (int)(t & 1);
                        else if constexpr (MODE == MODE_FP64) s = fma(t.y, t.x, s);
                        else s = fmaf(t.y, t.x, s);
                    }
#pragma unroll
                    for (int off = 16; off >= 1; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
                }
                if (timed && tid == 0) { uint64_t t = clock64(); ph[6] += t - tp; tp = t; }
                if (lane == 0) {
                    // kernel value K(up, low) and, from the tables on binary
                    // input, eta = 2 - 2K with the correctly rounded 1 / eta
                    double kul, rinv = 0.0, eta;
                    bool curved;
                    if constexpr (MODE == MODE_BINARY || BITS) {
                        int dist = BITS ? s : up.len + low.len - 2 * s;
                        dist = dist < 0 ? 0 : dist;
                        kul = ktab[dist];
                        rinv = rtab[dist];
                        eta = etab[dist];
                        curved = __double_as_longlong(rinv) != 0;   // eta > 1e-12
                    } else {
                        if (A.kernel == KERNEL_RBF) {
                            if constexpr (MODE == MODE_FP64) {
                                // the fixed-point exp, as in the row pass
                                double d2 = up.nrm + low.nrm - 2.0 * s;
                                kul = kul_cached ? kul_c
                                                 : exp_neg_fx(A.gamma * dpos(d2), expfx_s);
                            } else {
                                float d2 = (float)up.nrm + (float)low.nrm - 2.0f * s;
                                kul = (double)__expf(-gammaf * fmaxf(d2, 0.f));
                            }
                            eta = 2.0 - 2.0 * kul;   // K(x,x) = 1
                        } else {
                            // eta = K_uu + K_ll - 2 K_ul, K_uu from ||x_up||^2
                            double kuu, kll;
                            if constexpr (MODE == MODE_FP64) {
                                kul = kul_cached ? kul_c : kernel_of_dot(A.kernel, A.gamma, A.coef0, A.degree, s);
                                kuu = kernel_of_dot(A.kernel, A.gamma, A.coef0, A.degree, up.nrm);
                                kll = kernel_of_dot(A.kernel, A.gamma, A.coef0, A.degree, low.nrm);
                            } else {
                                const float c0 = (float)A.coef0;
                                kul = (double)kernel_of_dot(A.kernel, gammaf, c0, A.degree, (float)s);
                                kuu = (double)kernel_of_dot(A.kernel, gammaf, c0, A.degree, (float)up.nrm);
                                kll = (double)kernel_of_dot(A.kernel, gammaf, c0, A.degree, (float)low.nrm);
                            }
                            eta = __dsub_rn(__dadd_rn(kuu, kll), __dmul_rn(2.0, kul));
                        }
                        curved = dless(1e-12, eta);
                    }
                    // Eq. (alphaup) with rho = -eta (Eq. rho), K(x,x) = 1,
                    // clipped to the feasible segment [L, H]; end-point rule
                    // for a flat curvature. Each FP64 operation is the
                    // oracle's (same operands, same order). On this part a
                    // warp's FP64 instructions issue about one per 64 cycles,
                    // so signs y = +-1 are applied by choosing operands, and
                    // comparisons, clamps and snaps work on integer keys.
                    const bool yu_neg = up.y < 0, yl_neg = low.y < 0;
                    const double au = up.a, al = low.a;
                    const bool opposite = yu_neg != yl_neg;
                    // slope = y_low (f_up - f_low)
                    const double slope = (yl_neg ? low.f : up.f) - (yl_neg ? up.f : low.f);
                    // [L, H]: opposite labels L = max(0, al - au),
                    // H = min(C, (C + al) - au); equal labels L = max(0,
                    // (al + au) - C), H = min(C, al + au)
                    const double v1 = al + (opposite ? neg_if(au, true) : au);
                    const double w = (opposite ? C : v1) + (opposite ? al : neg_if(C, true));
                    const double h3 = w - au;
                    const double xL = opposite ? v1 : w, xH = opposite ? h3 : v1;
                    const double Lo = dless(xL, 0.0) ? 0.0 : xL;
                    const double Hi = dless(xH, C) ? xH : C;
                    double alc;
                    if (curved) {
                        double q;
                        if constexpr (MODE == MODE_BINARY || BITS) {
                            // slope / eta from the correctly rounded 1/eta of
                            // the table: one Markstein correction gives the
                            // correctly rounded quotient
                            const double q0 = slope * rinv;
                            const double r = fma(-eta, q0, slope);
                            q = fma(r, rinv, q0);
                        } else {
                            q = slope / eta;
                        }
                        const double t = al + q;
                        const unsigned long long kt = dkey(t);
                        alc = kt < dkey(Lo) ? Lo : (dkey(Hi) < kt ? Hi : t);
                    } else {
                        alc = dless(0.0, slope) ? Hi : Lo;
                    }
                    // alpha_up' = au + s (al - alpha_low'), s = y_up y_low,
                    // from the clipped (not yet snapped) alpha_low'
                    const double aunc = fma(opposite ? -1.0 : 1.0, al - alc, au);
                    const unsigned long long ka = dkey(alc), ku = dkey(aunc);
                    const unsigned long long ks = dkey(snap), kc = dkey(c_snap);
                    const double aln = ka < ks ? 0.0 : (kc < ka ? C : alc);
                    const double aun = ku < ks ? 0.0 : (kc < ku ? C : aunc);
                    // y_up (alpha_up' - au) and y_low (alpha_low' - al)
                    sh.du = (yu_neg ? au : aun) - (yu_neg ? aun : au);
                    sh.dl = (yl_neg ? al : aln) - (yl_neg ? aln : al);
                    sh.au_new = aun;
                    sh.al_new = aln;
                    sh.st_u = status_of(!yu_neg, aun, C);
                    sh.st_l = status_of(!yl_neg, aln, C);
                }
                __syncwarp();
                if constexpr (BITS && RES) step_bar_sync(kThreads);   // warp 0 joins the f updates
                else step_bar_arrive(kThreads);
                if (timed && tid == 0) { uint64_t t = clock64(); ph[1] += t - tp; tp = t; }
            }
        } else if constexpr (BITS && RES) {
            // ---- 3. row pass, bit-mask rows held on chip, in two sweeps
            //         over the active list: the squared distances of every
            //         row to x_up and x_low (warps 1..) while warp 0 runs the
            //         pair step, then, after a barrier of all warps, the FP64
            //         f updates (Eq. fup), the shrink rule and the candidates
            //         (all warps, below).
            if (!first) {
                for (int k = tid - 32; k < cnt; k += kThreads - 32) {
                    const uint4 *rb = bits_s + (size_t)act_s[k] * W4;
                    int du2 = 0, dl2 = 0;
#pragma unroll
                    for (int q = 0; q < W4; ++q) {
                        const uint4 v = rb[q];
                        du2 += __popc(v.x ^ up.m[4 * q]) + __popc(v.y ^ up.m[4 * q + 1]) +
                               __popc(v.z ^ up.m[4 * q + 2]) + __popc(v.w ^ up.m[4 * q + 3]);
                        dl2 += __popc(v.x ^ low.m[4 * q]) + __popc(v.y ^ low.m[4 * q + 1]) +
                               __popc(v.z ^ low.m[4 * q + 2]) + __popc(v.w ^ low.m[4 * q + 3]);
                    }
                    dist_s[k] = (uint32_t)du2 | ((uint32_t)dl2 << 16);
                }
                step_bar_sync(kThreads);
            }
        } else {
            // ---- 3. row pass over the segment's active list (warps 1..)
            constexpr int RPW = 32 / LPR;
            constexpr int kRowWarps = kWarps - 1;
            const int gl = lane & (LPR - 1);
            const int gw = lane / LPR;
            // kernel-row cache rows of this step (both found: no row sums)
            const bool kc_step = kc_on && !first;
            const bool kc_hu = kc_step && sh.kc_hu, kc_hl = kc_step && sh.kc_hl;
            KT *kc_ru = kc_step ? static_cast<KT *>(A.kc) + (size_t)sh.kc_su * A.kc_ld : nullptr;
            KT *kc_rl = kc_step ? static_cast<KT *>(A.kc) + (size_t)sh.kc_sl * A.kc_ld : nullptr;
            const bool skip_sums = kc_hu && kc_hl;
            const float up_nrmf = (float)up.nrm, low_nrmf = (float)low.nrm;
            // streamed segment with no row shrunk: its active list is the
            // identity (lists are reset to it and compacted in order), so the
            // row index needs no load
            const bool ident = !RES && cnt == nseg;
            double du = 0.0, dl = 0.0, au_new = 0.0, al_new = 0.0;
            unsigned char st_u = 0, st_l = 0;
            bool have_step = first;
            bool tiles_done = false;
            if constexpr (MODE == MODE_MIXED && LPR == 16) {
                if (A.dmat != nullptr && !kc_on) {
                    // Kernel rows on the tensor cores (mixed mode, RBF): tiles
                    // of 16 active rows x the two target rows (mma m16n8k16,
                    // BF16 inputs, FP32 accumulation; B columns 2..7 zero),
                    // rows read as dense BF16 from the d_pad-wide copy. Inside
                    // each 32-column block the K order is permuted so that a
                    // lane reads 8 consecutive values of a row with one
                    // 16-byte load: in k-step h of block b, logical k = 2t + i
                    // is column 32b + 8t + 4h + i and k = 2t + 8 + i column
                    // 32b + 8t + 4h + 2 + i; the targets use the same map, so
                    // the dot products are those of the rows. Each warp takes
                    // 32 active rows (two tiles) at a time and hands each
                    // row's two sums to one lane, which finishes the row as
                    // the CUDA-core pass does.
                    tiles_done = true;
                    const int g = lane >> 2, t4 = lane & 3;
                    const int nblk = A.d_pad >> 5;
                    uint2 *frag = reinterpret_cast<uint2 *>(dsm + L.frag);   // [2 nblk k-steps][32 lanes]
                    if (warp == 1) {
                        for (int ks = 0; ks < 2 * nblk; ++ks) {
                            const int b = ks >> 1, h = ks & 1;
                            uint32_t w0 = 0, w1 = 0;
                            if (!first && g < 2) {
                                const int c = 32 * b + 8 * t4 + 4 * h;
                                float e[4];
#pragma unroll
                                for (int x = 0; x < 4; ++x) {
                                    const int cx = c + x;
                                    e[x] = cx < d ? (g == 0 ? T[cx].x : T[cx].y) : 0.f;
                                }
                                const __nv_bfloat162 p0 = __floats2bfloat162_rn(e[0], e[1]);
                                const __nv_bfloat162 p1 = __floats2bfloat162_rn(e[2], e[3]);
                                w0 = *reinterpret_cast<const uint32_t *>(&p0);
                                w1 = *reinterpret_cast<const uint32_t *>(&p1);
                            }
                            frag[ks * 32 + lane] = make_uint2(w0, w1);
                        }
                    }
                    rows_bar_sync();
                    for (int base = (warp - 1) * 32;; base += kRowWarps * 32) {   // warp-uniform
                        const bool round0 = base == (warp - 1) * 32;
                        if (!round0 && base >= cnt) break;
                        float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
                        if (!first) {
#pragma unroll
                            for (int q = 0; q < 2; ++q) {
                                const int ka = base + 16 * q + g, kb2 = ka + 8;
                                const __nv_bfloat16 *pa = nullptr, *pb = nullptr;
                                if (ka < cnt) pa = A.dmat + (size_t)(lo + (ident ? ka : ACT(ka))) * A.d_pad + 8 * t4;
                                if (kb2 < cnt) pb = A.dmat + (size_t)(lo + (ident ? kb2 : ACT(kb2))) * A.d_pad + 8 * t4;
                                for (int b = 0; b < nblk; ++b) {
                                    const uint4 u = pa ? __ldg(reinterpret_cast<const uint4 *>(pa + 32 * b)) : make_uint4(0, 0, 0, 0);
                                    const uint4 v = pb ? __ldg(reinterpret_cast<const uint4 *>(pb + 32 * b)) : make_uint4(0, 0, 0, 0);
                                    const uint2 f0 = frag[(2 * b) * 32 + lane], f1 = frag[(2 * b + 1) * 32 + lane];
                                    mma_bf16_16816(acc[q], u.x, v.x, u.y, v.y, f0.x, f0.y);
                                    mma_bf16_16816(acc[q], u.z, v.z, u.w, v.w, f1.x, f1.y);
                                }
                            }
                        }
                        // the sums of active-list position base + lane: tile
                        // lane >> 4, row (lane & 15), held by lane 4 (lane & 7)
                        // as (acc[2 s], acc[2 s + 1]), s = (lane >> 3) & 1
                        const int src = 4 * (lane & 7);
                        const int qq = lane >> 4, ss = (lane >> 3) & 1;
                        float su = 0.f, sl = 0.f;
#pragma unroll
                        for (int q = 0; q < 2; ++q) {
#pragma unroll
                            for (int s2 = 0; s2 < 2; ++s2) {
                                const float a = __shfl_sync(0xffffffffu, acc[q][2 * s2], src);
                                const float b = __shfl_sync(0xffffffffu, acc[q][2 * s2 + 1], src);
                                if (q == qq && s2 == ss) { su = a; sl = b; }
                            }
                        }
                        const int k = base + lane;
                        const bool valid = k < cnt;
                        int r = 0;
                        double fi = 0.0;
                        uint8_t sb = 0;
                        double ku = 0.0, kl = 0.0;
                        if (valid) {
                            r = ident ? k : ACT(k);
                            fi = GETF(r);
                            sb = GETST(r);
                            if (!first) {
                                // K(x, x) = 1 exactly for the pair's own rows (the
                                // tile sums and the stored norms are summed in
                                // different orders, so their difference is not 0)
                                const int i = (int)(lo + r);
                                const float nrr = NRMF(r);
                                ku = i == up.i ? 1.0 : widen_f32(__expf(-gammaf * fmaxf(up_nrmf + nrr - 2.0f * su, 0.f)));
                                kl = i == low.i ? 1.0 : widen_f32(__expf(-gammaf * fmaxf(low_nrmf + nrr - 2.0f * sl, 0.f)));
                            }
                        }
                        if (!have_step) {
                            step_bar_sync(kThreads);
                            du = sh.du; dl = sh.dl;
                            st_u = sh.st_u; st_l = sh.st_l;
                            au_new = sh.au_new; al_new = sh.al_new;
                            have_step = true;
                        }
                        if (valid) {
                            const int i = (int)(lo + r);
                            if (!first) {
                                // Eq. (fup), FP64 accumulation
                                fi = fma(dl, kl, fma(du, ku, fi));
                                PUTF(r, fi);
                                if (i == up.i) {
                                    sb = st_u;
                                    PUTST(r, sb);
                                    PUTA(r, au_new);
                                } else if (i == low.i) {
                                    sb = st_l;
                                    PUTST(r, sb);
                                    PUTA(r, al_new);
                                }
                            }
                            const uint8_t set = set_bits(sb);
                            bool keep = true;
                            if (shrink_now) {
                                // Eq. (shrink), with the thresholds that chose this pair
                                keep = !(((set == ST_I3 || set == ST_I4) && dless(fi, bup_sel)) ||
                                         ((set == ST_I1 || set == ST_I2) && dless(blow_sel, fi)));
                                if (!keep) SET_ACT(k, ~r);
                            }
                            if (keep) {
                                const unsigned long long kup = key_up(fi), klo = key_low(fi);
                                // a lane meets its rows in increasing index order
                                if (st_up(set) && kup < bku) { bku = kup; biu = i; bru = r; }
                                if (st_low(set) && klo < bkl) { bkl = klo; bil = i; brl = r; }
                            }
                        }
                    }
                }
            }
            if (!tiles_done)
            for (int kb = (warp - 1) * RPW;; kb += kRowWarps * RPW) {
                const bool round0 = kb == (warp - 1) * RPW;
                if (!round0 && kb >= cnt) break;
                const int k = kb + gw;
                const bool valid = k < cnt;
                int r = 0;
                int64_t p0 = 0, p1 = 0;
                double fi = 0.0;
                uint8_t sb = 0;
                double nr = 0.0;
                float nrf = 0.f;
                if (valid) {
                    r = ident ? k : ACT(k);
                    if constexpr (!BITS) ROWP(r, p0, p1);
                    if (gl == 0) {
                        fi = GETF(r);
                        sb = GETST(r);
                        // issued with the row's other loads
                        if constexpr (!RES && MODE == MODE_MIXED) nrf = NRMF(r);
                        else if constexpr (!RES) nr = NRM(r);
                    }
                }
                Acc su = 0, sl = 0;
                if (xd && !first && !skip_sums) {
                    if constexpr (MODE == MODE_FP64) {
                        // exact inner products in integer arithmetic, each
                        // lane loading its next XB entries at once (4: fewer
                        // live registers than 8, measured 3% faster)
                        const int4 *T4 = reinterpret_cast<const int4 *>(T);
                        XdAcc au = xd_zero(), al = xd_zero();
                        constexpr int XB = 4;
                        for (int64_t pb = p0 + gl; pb < p1; pb += XB * LPR) {
                            int cb[XB];
                            uint32_t ub[XB];
#pragma unroll
                            for (int j = 0; j < XB; ++j) {
                                const int64_t p = pb + (int64_t)j * LPR;
                                cb[j] = 0;
                                ub[j] = 0u;
                                if (p < p1) XCW(p, cb[j], ub[j]);
                            }
#pragma unroll
                            for (int j = 0; j < XB; ++j) {
                                if (pb + (int64_t)j * LPR >= p1) break;
                                const int32_t m = xd_word_m(ub[j]);
                                const int e = xd_word_e(ub[j]);
                                const int4 t = T4[cb[j]];
                                xd_add(au, m, t.x, e + t.y);
                                xd_add(al, m, t.z, e + t.w);
                            }
                        }
                        xd_lane_sum<LPR>(au);
                        xd_lane_sum<LPR>(al);
                        su = xd_round(au, xd_unit);
                        sl = xd_round(al, xd_unit);
                    }
                } else if constexpr (BITS) {
                    // squared distances to x_up and x_low (one lane per row)
                    if (!first && valid) {
                        const uint4 *rb = RES ? bits_s + (size_t)r * W4 : bits_g + (size_t)(lo + r) * W4;
#pragma unroll
                        for (int q = 0; q < W4; ++q) {
                            const uint4 v = RES ? rb[q] : __ldg(rb + q);
                            su += __popc(v.x ^ up.m[4 * q]) + __popc(v.y ^ up.m[4 * q + 1]) +
                                  __popc(v.z ^ up.m[4 * q + 2]) + __popc(v.w ^ up.m[4 * q + 3]);
                            sl += __popc(v.x ^ low.m[4 * q]) + __popc(v.y ^ low.m[4 * q + 1]) +
                                  __popc(v.z ^ low.m[4 * q + 2]) + __popc(v.w ^ low.m[4 * q + 3]);
                        }
                    }
                } else if (!RES && !first && !skip_sums) {
                    // streamed rows: each lane loads its next 8 entries at once
                    // (one memory round trip per 8 entries, not one per entry;
                    // mixed rows one word per entry when packed)
                    for (int64_t pb = p0 + gl; pb < p1; pb += 8 * LPR) {
                        int cb[8];
                        float vb[8];
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const int64_t p = pb + (int64_t)j * LPR;
                            const bool in = p < p1;
                            if constexpr (MODE == MODE_MIXED) {
                                if (A.ew) {
                                    // mixed rows packed one word per entry (d < 2^16)
                                    const uint32_t w = in ? A.ew[p] : 0u;
                                    cb[j] = (int)(w & 0xffffu);
                                    vb[j] = __uint_as_float(w & 0xffff0000u);
                                } else {
                                    cb[j] = in ? COL(p) : 0;
                                    vb[j] = in ? VAL(p) : 0.f;
                                }
                            } else {
                                cb[j] = in ? COL(p) : 0;
                                if constexpr (MODE != MODE_BINARY) vb[j] = in ? VAL(p) : 0.f;
                            }
                        }
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            if (pb + (int64_t)j * LPR >= p1) break;
                            if constexpr (MODE == MODE_BINARY) {
                                unsigned short t = T[cb[j]];
                                su += (int)(t & 0xff);
                                sl += (int)(t >> 8);
                            } else if constexpr (MODE == MODE_FP64) {
                                double2 t = T[cb[j]];
                                const double v = widen_f32(vb[j]);
                                su = fma(v, t.x, su);
                                sl = fma(v, t.y, sl);
                            } else {
                                float2 t = T[cb[j]];
                                su = fmaf(vb[j], t.x, su);
                                sl = fmaf(vb[j], t.y, sl);
                            }
                        }
                    }
#pragma unroll
                    for (int off = LPR / 2; off >= 1; off >>= 1) {
                        su += __shfl_xor_sync(0xffffffffu, su, off);
                        sl += __shfl_xor_sync(0xffffffffu, sl, off);
                    }
                } else if (!first && !skip_sums) {
                    for (int64_t p = p0 + gl; p < p1; p += LPR) {
                        const int c = COL(p);
                        if constexpr (MODE == MODE_BINARY) {
                            unsigned short t = T[c];
                            su += (int)(t & 0xff);
                            sl += (int)(t >> 8);
                        } else if constexpr (MODE == MODE_FP64) {
                            const double v = widen_f32(VAL(p));
                            double2 t = T[c];
                            su = fma(v, t.x, su);
                            sl = fma(v, t.y, sl);
                        } else {
                            float v = VAL(p);
                            float2 t = T[c];
                            su = fmaf(v, t.x, su);
                            sl = fmaf(v, t.y, sl);
                        }
                    }
#pragma unroll
                    for (int off = LPR / 2; off >= 1; off >>= 1) {
                        su += __shfl_xor_sync(0xffffffffu, su, off);
                        sl += __shfl_xor_sync(0xffffffffu, sl, off);
                    }
                }
                double ku = 0.0, kl = 0.0;
                if (!first && valid && gl == 0) {
                    const int len = (int)(p1 - p0);
                    if constexpr (BITS) {
                        ku = ktab[su];
                        kl = ktab[sl];
                    } else if constexpr (MODE == MODE_BINARY) {
                        int du2 = up.len + len - 2 * su, dl2 = low.len + len - 2 * sl;
                        ku = ktab[du2 < 0 ? 0 : du2];
                        kl = ktab[dl2 < 0 ? 0 : dl2];
                    } else {
                        const int64_t gi = lo + r;
                        if constexpr (MODE == MODE_FP64) {
                            const double nrr = RES ? NRM(r) : nr;
                            if (kc_hu) {
                                ku = kc_ru[gi];
                            } else {
                                if (A.kernel != KERNEL_RBF) {
                                    ku = kernel_of_dot(A.kernel, A.gamma, A.coef0, A.degree, (double)su);
                                } else {
                                    const double d2u = up.nrm + nrr - 2.0 * su;
                                    ku = exp_neg_fx(A.gamma * dpos(d2u), expfx_s);
                                }
                                if (kc_step) kc_ru[gi] = ku;
                            }
                            if (kc_hl) {
                                kl = kc_rl[gi];
                            } else {
                                if (A.kernel != KERNEL_RBF) {
                                    kl = kernel_of_dot(A.kernel, A.gamma, A.coef0, A.degree, (double)sl);
                                } else {
                                    const double d2l = low.nrm + nrr - 2.0 * sl;
                                    kl = exp_neg_fx(A.gamma * dpos(d2l), expfx_s);
                                }
                                if (kc_step) kc_rl[gi] = kl;
                            }
                        } else {
                            // mixed: FP32 kernel values, widened exactly for
                            // the FP64 f update by integer operations
                            const float nrr = RES ? NRMF(r) : nrf;
                            float kuf, klf;
                            if (kc_hu) {
                                kuf = kc_ru[gi];
                            } else {
                                if (A.kernel != KERNEL_RBF)
                                    kuf = kernel_of_dot(A.kernel, gammaf, (float)A.coef0, A.degree, (float)su);
                                else
                                    kuf = __expf(-gammaf * fmaxf(up_nrmf + nrr - 2.0f * su, 0.f));
                                if (kc_step) kc_ru[gi] = kuf;
                            }
                            if (kc_hl) {
                                klf = kc_rl[gi];
                            } else {
                                if (A.kernel != KERNEL_RBF)
                                    klf = kernel_of_dot(A.kernel, gammaf, (float)A.coef0, A.degree, (float)sl);
                                else
                                    klf = __expf(-gammaf * fmaxf(low_nrmf + nrr - 2.0f * sl, 0.f));
                                if (kc_step) kc_rl[gi] = klf;
                            }
                            ku = widen_f32(kuf);
                            kl = widen_f32(klf);
                        }
                    }
                }
                if (!have_step) {
                    step_bar_sync(kThreads);
                    du = sh.du; dl = sh.dl;
                    st_u = sh.st_u; st_l = sh.st_l;
                    au_new = sh.au_new; al_new = sh.al_new;
                    have_step = true;
                }
                if (valid && gl == 0) {
                    const int i = (int)(lo + r);
                    if (!first) {
                        // Eq. (fup), FP64 accumulation
                        fi = fma(dl, kl, fma(du, ku, fi));
                        PUTF(r, fi);
                        if (i == up.i) {
                            sb = st_u;
                            PUTST(r, sb);
                            PUTA(r, au_new);
                        } else if (i == low.i) {
                            sb = st_l;
                            PUTST(r, sb);
                            PUTA(r, al_new);
                        }
                    }
                    const uint8_t set = set_bits(sb);
                    bool keep = true;
                    if (shrink_now) {
                        // Eq. (shrink), with the thresholds that chose this pair
                        keep = !(((set == ST_I3 || set == ST_I4) && dless(fi, bup_sel)) ||
                                 ((set == ST_I1 || set == ST_I2) && dless(blow_sel, fi)));
                        if (!keep) SET_ACT(k, ~r);
                    }
                    if (keep) {
                        const unsigned long long kup = key_up(fi), klo = key_low(fi);
                        // a thread meets its rows in increasing index order:
                        // a strict key test keeps the lowest index of a tie
                        if (st_up(set) && kup < bku) { bku = kup; biu = i; bru = r; }
                        if (st_low(set) && klo < bkl) { bkl = klo; bil = i; brl = r; }
                    }
                }
            }
        }
        if constexpr (BITS && RES) {
            // second sweep, all warps: f updates, shrink rule, candidates
            const double du = sh.du, dl = sh.dl, au_new = sh.au_new, al_new = sh.al_new;
            const unsigned char st_u = sh.st_u, st_l = sh.st_l;
            for (int k = tid; k < cnt; k += kThreads) {
                const int r = act_s[k];
                const int i = (int)(lo + r);
                double fi = f_s[r];
                uint8_t sb = st_s[r];
                if (!first) {
                    const uint32_t dd = dist_s[k];
                    fi = fma(dl, ktab[dd >> 16], fma(du, ktab[dd & 0xffffu], fi));
                    f_s[r] = fi;
                    if (i == up.i) {
                        sb = st_u;
                        st_s[r] = sb;
                        a_s[r] = au_new;
                    } else if (i == low.i) {
                        sb = st_l;
                        st_s[r] = sb;
                        a_s[r] = al_new;
                    }
                }
                const uint8_t set = set_bits(sb);
                bool keep = true;
                if (shrink_now) {
                    keep = !(((set == ST_I3 || set == ST_I4) && dless(fi, bup_sel)) ||
                             ((set == ST_I1 || set == ST_I2) && dless(blow_sel, fi)));
                    if (!keep) act_s[k] = ~r;
                }
                if (keep) {
                    const unsigned long long kup = key_up(fi), klo = key_low(fi);
                    // increasing index order per thread: strict key test
                    if (st_up(set) && kup < bku) { bku = kup; biu = i; bru = r; }
                    if (st_low(set) && klo < bkl) { bkl = klo; bil = i; brl = r; }
                }
            }
        }
        // payload of a segment row for the exchange (read after this
        // thread's own updates of f, alpha and the index set)
        auto make_side = [&](int r) {
            Side sd;
            int64_t p0 = 0, p1 = 0;
            if constexpr (!BITS) ROWP(r, p0, p1);
            const uint8_t sb = GETST(r);
            sd.f = GETF(r);
            sd.a = GETA(r);
            sd.nrm = NRM(r);
            sd.p0 = RES ? base + p0 : p0;
            sd.i = (int)(lo + r);
            sd.len = (int)(p1 - p0);
            sd.y = y_of(sb);
            sd.owner = cid;
#pragma unroll
            for (int w = 0; w < 8; ++w) sd.m[w] = 0;
            if constexpr (BITS) {
                const uint4 *rb = RES ? bits_s + (size_t)r * W4 : bits_g + (size_t)(lo + r) * W4;
#pragma unroll
                for (int q = 0; q < W4; ++q) {
                    const uint4 v = rb[q];
                    sd.m[4 * q] = v.x; sd.m[4 * q + 1] = v.y; sd.m[4 * q + 2] = v.z; sd.m[4 * q + 3] = v.w;
                }
            }
            return sd;
        };
        // ---- CTA reduction: warp minima of (key, index); winners' payloads.
        //      Gain exchange (gx): both sides are the gain winner's row, the
        //      I_up side carrying -gain in place of f as its key.
        auto cta_reduce = [&](bool gx, unsigned long long ku_, int iu_, int ru_, unsigned long long kl_,
                              int il_, int rl_, double gneg) {
            unsigned long long k1 = ku_, k2 = kl_;
            int i1 = iu_, i2 = il_;
            warp_min_ki(k1, i1);
            warp_min_ki(k2, i2);
            if (lane == 0) {
                sh.wkup[warp] = k1; sh.wiup[warp] = i1;
                sh.wklow[warp] = k2; sh.wilow[warp] = i2;
            }
            if (i1 != INT_MAX && iu_ == i1) {
                Side sd = make_side(ru_);
                if (gx) sd.f = gneg;
                sh.wup[warp] = sd;
            }
            if (i2 != INT_MAX && il_ == i2) sh.wlow[warp] = make_side(rl_);
            __syncthreads();
        };
        cta_reduce(false, bku, biu, bru, bkl, bil, brl, 0.0);
        // ---- 5. compaction of the active list on shrink steps
        if (shrink_now) {
            int kept = 0;
            for (int b0 = 0; b0 < cnt; b0 += kThreads) {
                int k = b0 + tid;
                int v = k < cnt ? ACT(k) : -1;
                bool keepv = v >= 0;
                int pos = block_scan_flag(keepv, sh.scan, &sh.scan_tot);
                int tot = sh.scan_tot;
                if (keepv) SET_ACT(kept + pos, v);
                kept += tot;
                __syncthreads();
            }
            cnt = kept;
        }
        if (timed && tid == 0) { uint64_t t = clock64(); ph[2] += t - tp; tp = t; }
        // tagged slot of the exchange through global memory, per leader (per
        // CTA in a flat launch) and epoch parity
        auto tslot = [&](int par, int c) {
            return reinterpret_cast<ulonglong2 *>(static_cast<unsigned char *>(A.cand) + ((size_t)par * nlead + c) * kCandStride);
        };
        auto exchange = [&](bool gx) {
            // ---- 4. grid-wide exchange. One cluster over the whole grid: each
            //         CTA writes its candidate into every CTA's shared memory and
            //         arrives on that CTA's mbarrier; every CTA reduces the same
            //         candidates in the same order. Several clusters: the CTAs of a
            //         cluster hand their candidates to its first CTA through
            //         distributed shared memory; only those leaders exchange
            //         through global memory (tagged slots when one warp polls
            //         them all, else a release/acquire flag per slot; bounded
            //         waits) and push the result back to their cluster.
            ++epoch;
            const int par = (int)(epoch & 1);
            const int phs = gx ? 7 : 3;
            if (warp == 0) {
                unsigned long long k1 = lane < kWarps ? sh.wkup[lane] : kNoKey;
                unsigned long long k2 = lane < kWarps ? sh.wklow[lane] : kNoKey;
                int i1 = lane < kWarps ? sh.wiup[lane] : INT_MAX;
                int i2 = lane < kWarps ? sh.wilow[lane] : INT_MAX;
                const unsigned long long k1s = k1, k2s = k2;
                const int i1s = i1, i2s = i2;
                warp_min_ki(k1, i1);
                warp_min_ki(k2, i2);
                const unsigned mu = __ballot_sync(0xffffffffu, i1 != INT_MAX && k1s == k1 && i1s == i1);
                const unsigned ml = __ballot_sync(0xffffffffu, i2 != INT_MAX && k2s == k2 && i2s == i2);
                if constexpr (solo) {
                    // lane q sends the CTA's candidate to CTA q: the winning
                    // warps' sides straight from shared memory, then the count
                    if (lane < csize) {
                        const uint32_t dst = cluster_addr(smem_u32(&sh.xc[par][crank]), lane);
                        const uint32_t rbar = cluster_addr(smem_u32(&sh.xbar[par]), lane);
                        const uint4 *su = reinterpret_cast<const uint4 *>(mu ? &sh.wup[__ffs(mu) - 1] : &sh.none[0]);
                        const uint4 *sl = reinterpret_cast<const uint4 *>(ml ? &sh.wlow[__ffs(ml) - 1] : &sh.none[1]);
                        constexpr int kSideV = (int)(sizeof(Side) / 16);
#pragma unroll
                        for (int j = 0; j < kSideV; ++j) st_async_v4(dst + 16 * j, su[j], rbar);
#pragma unroll
                        for (int j = 0; j < kSideV; ++j) st_async_v4(dst + (uint32_t)sizeof(Side) + 16 * j, sl[j], rbar);
                        st_async_v4(dst + (uint32_t)offsetof(CandFull, count), make_uint4((unsigned)cnt, 0u, 0u, 0u), rbar);
                    }
                    if (lane == 0)
                        mbar_arrive_expect_tx(smem_u32(&sh.xbar[par]), (uint32_t)(csize * sizeof(CandFull)));
                } else if (lane == 0) {
                    CandFull cf;
                    if (mu) cf.up = sh.wup[__ffs(mu) - 1]; else side_empty(cf.up, true);
                    if (ml) cf.low = sh.wlow[__ffs(ml) - 1]; else side_empty(cf.low, false);
                    cf.count = cnt;
                    cf.pad[0] = cf.pad[1] = cf.pad[2] = 0;
                    CandFull *dst = cluster.map_shared_rank(sh.ccand, 0);
                    dst[crank] = cf;
                }
                if (lane == 0) {
                    if (busy_on) busy += clock64() - cta_t0;
                    if (timed) { uint64_t t = clock64(); ph[phs] += t - tp; tp = t; }
                }
            }
            // the previous step's target rows are cleared while others wait
            if (!BITS && !gx && prev_valid && warp >= 8) {
                Tgt *P = tbuf + (size_t)(1 - buf) * d;
                const int *pcu = tcol + (size_t)((1 - buf) * 2 + 0) * maxnnz;
                const int *pcl = tcol + (size_t)((1 - buf) * 2 + 1) * maxnnz;
                for (int k = tid - 256; k < prev_len_u; k += kThreads - 256) P[pcu[k]] = tclear;
                for (int k = tid - 256; k < prev_len_l; k += kThreads - 256) P[pcl[k]] = tclear;
            }
            if constexpr (solo) {
                if (warp == 0) {
                    // this epoch's csize candidates; the k-th use of a barrier
                    // completes its phase of parity k & 1
                    const uint32_t bar = smem_u32(&sh.xbar[par]);
                    const uint32_t parity = (uint32_t)((epoch - 1) >> 1) & 1u;
                    int timed_out = mbar_wait_bounded(bar, parity, A.timeout_ns, &A.ctrl->err);
                    timed_out = __any_sync(0xffffffffu, timed_out);
                    if (timed_out && lane == 0) atomicExch(&A.ctrl->err, 1);
                    unsigned long long k1 = kNoKey, k2 = kNoKey;
                    int i1 = INT_MAX, i2 = INT_MAX;
                    long long cc = 0;
                    if (lane < csize && !timed_out) cand_keys(sh.xc[par][lane], k1, i1, k2, i2, cc);
                    if (gx) { k2 = k1; i2 = i1; }   // the gain winner's row on both sides
                    const unsigned long long k1s = k1, k2s = k2;
                    const int i1s = i1, i2s = i2;
                    warp_min_ki(k1, i1);
                    warp_min_ki(k2, i2);
#pragma unroll
                    for (int off = 16; off >= 1; off >>= 1) cc += __shfl_xor_sync(0xffffffffu, cc, off);
                    const unsigned mu = __ballot_sync(0xffffffffu, i1 != INT_MAX && k1s == k1 && i1s == i1);
                    const unsigned ml = __ballot_sync(0xffffffffu, i2 != INT_MAX && k2s == k2 && i2s == i2);
                    // the winning sides into the result, one 8-byte word per lane
                    const Side *wsu = mu ? &sh.xc[par][__ffs(mu) - 1].up : &sh.none[0];
                    const Side *wsl = ml ? &sh.xc[par][__ffs(ml) - 1].low : &sh.none[1];
                    constexpr int kSideW = (int)(sizeof(Side) / 8);
                    static_assert(2 * kSideW <= 32, "a side is copied by one warp");
                    if (lane < 2 * kSideW) {
                        const bool u = lane < kSideW;
                        const int w = u ? lane : lane - kSideW;
                        reinterpret_cast<unsigned long long *>(u ? &sh.res.up : &sh.res.low)[w] =
                            reinterpret_cast<const unsigned long long *>(u ? wsu : wsl)[w];
                    }
                    if (lane == 0) {
                        sh.res.total = cc;
                        sh.res.flag = timed_out;
                        sh.res.gap_open = dless(A.thr, wsl->f - wsu->f);
                    }
                }
                __syncthreads();
            } else {
                cluster.sync();
                const int rwarps = xwarps;
                // FP64 with the kernel-row cache: each CTA reads K(up, low)
                // of a cached row from the entry another CTA wrote. Each
                // leader releases the epoch (its cluster's writes before the
                // barrier above) on a flag of its own, and every CTA records
                // the least epoch it sees released by all leaders, both by
                // warps that have no part in the exchange.
                const bool rel_on = MODE == MODE_FP64 && kc_on;
                if (rel_on && warp > rwarps) {
                    unsigned m = 0xffffffffu;
                    for (int c = (warp - rwarps - 1) * 32 + lane; c < nlead; c += (kWarps - rwarps - 1) * 32)
                        m = min(m, ld_acquire_u32(rel_flag(c)));
                    m = __reduce_min_sync(0xffffffffu, m);
                    if (lane == 0) sh.rrel[warp] = m;
                }
                if (crank == 0) {
                    if (warp == 0) {
                        // cluster winner -> this leader's global slot
                        unsigned long long k1 = kNoKey, k2 = kNoKey;
                        int i1 = INT_MAX, i2 = INT_MAX;
                        long long cc = 0;
                        if (lane < csize) cand_keys(sh.ccand[lane], k1, i1, k2, i2, cc);
                        if (gx) { k2 = k1; i2 = i1; }
                        const unsigned long long k1s = k1, k2s = k2;
                        const int i1s = i1, i2s = i2;
                        warp_min_ki(k1, i1);
                        warp_min_ki(k2, i2);
#pragma unroll
                        for (int off = 16; off >= 1; off >>= 1) cc += __shfl_xor_sync(0xffffffffu, cc, off);
                        const unsigned mu = __ballot_sync(0xffffffffu, i1 != INT_MAX && k1s == k1 && i1s == i1);
                        const unsigned ml = __ballot_sync(0xffffffffu, i2 != INT_MAX && k2s == k2 && i2s == i2);
                        if (!tagged) {
                            if (lane == 0) {
                                CandFull *out = reinterpret_cast<CandFull *>(static_cast<unsigned char *>(A.cand) +
                                                                             ((size_t)par * nlead + cid) * kCandStride);
                                if (mu) copy_side(&out->up, &sh.ccand[__ffs(mu) - 1].up);
                                else { Side e; side_empty(e, true); copy_side(&out->up, &e); }
                                if (ml) copy_side(&out->low, &sh.ccand[__ffs(ml) - 1].low);
                                else { Side e; side_empty(e, false); copy_side(&out->low, &e); }
                                out->count = (int32_t)cc;
                                st_release_u32(A.seq + ((size_t)par * nlead + cid) * kSeqStride, epoch);
                            }
                        } else if (lane < kTagPairs) {
                            // the first 48 bytes of both winning sides and the
                            // count, as tagged words (lane j: words 2j, 2j + 1)
                            const uint32_t *wsu = reinterpret_cast<const uint32_t *>(mu ? &sh.ccand[__ffs(mu) - 1].up : &sh.none[0]);
                            const uint32_t *wsl = reinterpret_cast<const uint32_t *>(ml ? &sh.ccand[__ffs(ml) - 1].low : &sh.none[1]);
                            auto word = [&](int q) -> uint32_t {
                                return q < 12 ? wsu[q] : (q < 24 ? wsl[q - 12] : (q == 24 ? (uint32_t)cc : 0u));
                            };
                            st_tagged2(tslot(par, cid) + lane, word(2 * lane), word(2 * lane + 1), epoch);
                        }
                    }
                    if (rel_on && warp == rwarps && lane == 0) st_release_u32(rel_flag(cid), epoch);
                    if (warp < rwarps) {
                        const int c = warp * 32 + lane;
                        int ai = INT_MAX, bi = INT_MAX;
                        double af = 0.0, bf = 0.0;
                        const CandFull *gp = nullptr;
                        long long cc = 0;
                        int timed_out = 0;
                        // the first 48 bytes of both sides (all but the bit
                        // masks), read with the keys: the winning lane then
                        // writes its side without another trip to L2
                        uint4 wu0 = make_uint4(0, 0, 0, 0), wu1 = wu0, wu2 = wu0, wl0 = wu0, wl1 = wu0, wl2 = wu0;
                        if (c < nlead) {
                            uint64_t t0 = 0;
                            int spins = 0;
                            auto waited_out = [&]() {
                                if (++spins >= 256) {
                                    spins = 0;
                                    uint64_t now = global_ns();
                                    if (t0 == 0) t0 = now;
                                    else if (now - t0 > (uint64_t)A.timeout_ns) return true;
                                    if (*(volatile int *)&A.ctrl->err) return true;
                                }
                                return false;
                            };
                            if (!tagged) {
                                const unsigned *sp = A.seq + ((size_t)par * nlead + c) * kSeqStride;
                                // acquire loads: the slot was written before the flag
                                while (ld_acquire_u32(sp) < epoch) {
                                    if (waited_out()) { timed_out = 1; break; }
                                }
                                if (!timed_out) {
                                    // L2 reads (bypass L1, which is not coherent across SMs)
                                    gp = reinterpret_cast<const CandFull *>(static_cast<const unsigned char *>(A.cand) +
                                                                            ((size_t)par * nlead + c) * kCandStride);
                                    const uint4 *pu = reinterpret_cast<const uint4 *>(&gp->up);
                                    const uint4 *pl = reinterpret_cast<const uint4 *>(&gp->low);
                                    wu0 = __ldcg(pu); wu1 = __ldcg(pu + 1); wu2 = __ldcg(pu + 2);
                                    wl0 = __ldcg(pl); wl1 = __ldcg(pl + 1); wl2 = __ldcg(pl + 2);
                                    cc = __ldcg(&gp->count);
                                }
                            } else {
                                // every word of the slot tagged with this epoch
                                const ulonglong2 *sp = tslot(par, c);
                                uint32_t d[2 * kTagPairs];
                                for (;;) {
                                    unsigned ok = 1u;
#pragma unroll
                                    for (int j = 0; j < kTagPairs; ++j) {
                                        const ulonglong2 w = ld_tagged2(sp + j);
                                        d[2 * j] = (uint32_t)w.x;
                                        d[2 * j + 1] = (uint32_t)w.y;
                                        ok &= (unsigned)((uint32_t)(w.x >> 32) == epoch) & (unsigned)((uint32_t)(w.y >> 32) == epoch);
                                    }
                                    if (ok) break;
                                    if (waited_out()) { timed_out = 1; break; }
                                }
                                if (!timed_out) {
                                    wu0 = make_uint4(d[0], d[1], d[2], d[3]);
                                    wu1 = make_uint4(d[4], d[5], d[6], d[7]);
                                    wu2 = make_uint4(d[8], d[9], d[10], d[11]);
                                    wl0 = make_uint4(d[12], d[13], d[14], d[15]);
                                    wl1 = make_uint4(d[16], d[17], d[18], d[19]);
                                    wl2 = make_uint4(d[20], d[21], d[22], d[23]);
                                    cc = (int)d[24];
                                }
                            }
                            if (!timed_out) {
                                ai = (int)wu2.x;
                                bi = (int)wl2.x;
                                af = __hiloint2double((int)wu0.y, (int)wu0.x);
                                bf = __hiloint2double((int)wl0.y, (int)wl0.x);
                            }
                        }
                        const int any_to = __any_sync(0xffffffffu, timed_out);
                        if (any_to && lane == 0) atomicExch(&A.ctrl->err, 1);
                        unsigned long long k1 = ai == INT_MAX ? kNoKey : key_up(af);
                        unsigned long long k2 = bi == INT_MAX ? kNoKey : key_low(bf);
                        int i1 = ai, i2 = bi;
                        if (gx) { k2 = k1; i2 = i1; }
                        warp_min_ki(k1, i1);
                        warp_min_ki(k2, i2);
#pragma unroll
                        for (int off = 16; off >= 1; off >>= 1) cc += __shfl_xor_sync(0xffffffffu, cc, off);
                        if (tagged) {
                            // one warp holds every leader's candidate: the
                            // winning sides go from their lanes straight into
                            // the result area of every CTA of the cluster
                            // (lane q writes CTA q's)
                            const unsigned mu = __ballot_sync(0xffffffffu, i1 != INT_MAX && ai == i1);
                            const unsigned ml = __ballot_sync(0xffffffffu, i2 != INT_MAX && bi == i2);
                            const int su = mu ? __ffs(mu) - 1 : 0, sl = ml ? __ffs(ml) - 1 : 0;
                            uint4 ru[3] = {shfl_u4(wu0, su), shfl_u4(wu1, su), shfl_u4(wu2, su)};
                            uint4 rl[3] = {shfl_u4(wl0, sl), shfl_u4(wl1, sl), shfl_u4(wl2, sl)};
                            if (!mu) {
                                const uint4 *e = reinterpret_cast<const uint4 *>(&sh.none[0]);
                                ru[0] = e[0]; ru[1] = e[1]; ru[2] = e[2];
                            }
                            if (!ml) {
                                const uint4 *e = reinterpret_cast<const uint4 *>(&sh.none[1]);
                                rl[0] = e[0]; rl[1] = e[1]; rl[2] = e[2];
                            }
                            const double fu = __hiloint2double((int)ru[0].y, (int)ru[0].x);
                            const double fl = __hiloint2double((int)rl[0].y, (int)rl[0].x);
                            const uint4 tail = make_uint4((unsigned)(unsigned long long)cc, (unsigned)((unsigned long long)cc >> 32),
                                                          (unsigned)any_to, (unsigned)dless(A.thr, fl - fu));
                            if (lane < csize) {
                                uint4 *o = reinterpret_cast<uint4 *>(cluster.map_shared_rank(&sh.res, lane));
                                o[0] = ru[0]; o[1] = ru[1]; o[2] = ru[2];
                                o[5] = rl[0]; o[6] = rl[1]; o[7] = rl[2];
                                o[10] = tail;
                            }
                        } else {
                            if (lane == 0) {
                                sh.rkup[warp] = k1; sh.riup[warp] = i1;
                                sh.rklow[warp] = k2; sh.rilow[warp] = i2;
                                sh.rcount[warp] = cc;
                                sh.rto[warp] = any_to;
                            }
                            if constexpr (BITS) {
                                if (i1 != INT_MAX && ai == i1) copy_side_ldcg(&sh.rup[warp], &gp->up);
                                if (i2 != INT_MAX && bi == i2) copy_side_ldcg(&sh.rlow[warp], &gp->low);
                            } else {
                                auto put48 = [](Side *dst, const uint4 &a, const uint4 &b, const uint4 &c) {
                                    unsigned long long *d8 = reinterpret_cast<unsigned long long *>(dst);
                                    const uint4 v[3] = {a, b, c};
#pragma unroll
                                    for (int w = 0; w < 3; ++w) {
                                        d8[2 * w] = ((unsigned long long)v[w].y << 32) | v[w].x;
                                        d8[2 * w + 1] = ((unsigned long long)v[w].w << 32) | v[w].z;
                                    }
                                };
                                if (i1 != INT_MAX && ai == i1) put48(&sh.rup[warp], wu0, wu1, wu2);
                                if (i2 != INT_MAX && bi == i2) put48(&sh.rlow[warp], wl0, wl1, wl2);
                            }
                        }
                    }
                    if (!tagged) {
                        __syncthreads();
                        if (warp == 0) {
                            // final winner, pushed to every CTA of the cluster
                            unsigned long long ku = sh.rkup[0], kl = sh.rklow[0];
                            int iu = sh.riup[0], il = sh.rilow[0], wu = 0, wl = 0, to = sh.rto[0];
                            long long cc = sh.rcount[0];
                            for (int w = 1; w < rwarps; ++w) {
                                if (ki_less(sh.rkup[w], sh.riup[w], ku, iu)) { ku = sh.rkup[w]; iu = sh.riup[w]; wu = w; }
                                if (ki_less(sh.rklow[w], sh.rilow[w], kl, il)) { kl = sh.rklow[w]; il = sh.rilow[w]; wl = w; }
                                cc += sh.rcount[w];
                                to |= sh.rto[w];
                            }
                            if (lane == 0) {
                                if (iu != INT_MAX) copy_side(&sh.res.up, &sh.rup[wu]); else side_empty(sh.res.up, true);
                                if (il != INT_MAX) copy_side(&sh.res.low, &sh.rlow[wl]); else side_empty(sh.res.low, false);
                                sh.res.total = cc;
                                sh.res.flag = to;
                                sh.res.gap_open = dless(A.thr, sh.res.low.f - sh.res.up.f);
                            }
                            __syncwarp();
                            if (lane > 0 && lane < csize) copy_result(cluster.map_shared_rank(&sh.res, lane), &sh.res);
                        }
                    }
                }
                cluster.sync();
            }
        };
        exchange(false);
        if (timed && tid == 0) { uint64_t t = clock64(); ph[4] += t - tp; tp = t; }
        if (sh.res.flag) break;
        prev_valid = first ? 0 : 1;
        prev_len_u = up.len;
        prev_len_l = low.len;
        up = sh.res.up;
        low = sh.res.low;
        total = sh.res.total;
        gap_open = sh.res.gap_open != 0;
        if (!first) {
            ++iter;
            if (shrink_now) {
                counter = A.h < total ? A.h : total;
                if (counter < 1) counter = 1;
                ++shrink_events;
                if (cta == 0 && tid == 0 && shrink_events <= A.atrace_len) {
                    A.atrace[2 * (shrink_events - 1)] = iter;
                    A.atrace[2 * (shrink_events - 1) + 1] = total;
                }
            }
        }
        first = false;
        if constexpr (WSS) {
            // ---- 6. second-order choice of x_low (the paper's future work,
            //         Section VI): over the active rows t of I_low with
            //         f_t > f_up, the largest gain (f_t - f_up)^2 / eta_ut,
            //         eta_ut = K_uu + K_tt - 2 K_ut (1e-12 when not positive),
            //         lowest index on ties; the first-order b_low stays the
            //         stopping test's and the shrink rule's. Runs only when
            //         another step follows.
            beta_low = low.f;
            if (gap_open && iter < A.iter_limit) {
                unsigned long long gk = kNoKey;   // dkey(-gain): larger gain, smaller key
                int gi = INT_MAX, gr = 0;
                double gneg = 0.0;
                auto consider = [&](double ft, double eta, int i, int r) {
                    const double b = ft - up.f;
                    const double a = dless(0.0, eta) ? eta : 1e-12;
                    const double g = __ddiv_rn(__dmul_rn(b, b), a);
                    const double ng = neg_if(g, true);
                    const unsigned long long key = dkey(ng);
                    // rows met in increasing index order: strict test keeps the lowest
                    if (key < gk) { gk = key; gi = i; gr = r; gneg = ng; }
                };
                const unsigned long long kfu = dkey(up.f);
                if constexpr (BITS) {
                    for (int k = tid; k < cnt; k += kThreads) {
                        const int r = ACT(k);
                        const uint8_t sb = GETST(r);
                        const double ft = GETF(r);
                        if (!st_low(set_bits(sb)) || !(kfu < dkey(ft))) continue;
                        const uint4 *rb = RES ? bits_s + (size_t)r * W4 : bits_g + (size_t)(lo + r) * W4;
                        int dist = 0;
#pragma unroll
                        for (int q = 0; q < W4; ++q) {
                            const uint4 v = RES ? rb[q] : __ldg(rb + q);
                            dist += __popc(v.x ^ up.m[4 * q]) + __popc(v.y ^ up.m[4 * q + 1]) +
                                    __popc(v.z ^ up.m[4 * q + 2]) + __popc(v.w ^ up.m[4 * q + 3]);
                        }
                        consider(ft, etab[dist], (int)(lo + r), r);
                    }
                } else {
                    // x_up into the next step's (clean) target buffer, as the
                    // next step's own fill will write it
                    Tgt *Tn = tbuf + (size_t)(iter & 1) * d;
                    for (int k = tid; k < up.len; k += kThreads) {
                        const int c = A.indices[up.p0 + k];
                        if constexpr (MODE == MODE_BINARY) reinterpret_cast<unsigned char *>(Tn + c)[0] = 1;
                        else if constexpr (MODE == MODE_FP64) xd_put<0>(Tn[c], A.values[up.p0 + k], xd, xd_tmin, xd_te);
                        else Tn[c].x = A.vmix[up.p0 + k];
                    }
                    __syncthreads();
                    double kuu = 0.0;   // K(x_up, x_up) of a non-RBF kernel
                    if (A.kernel != KERNEL_RBF) {
                        if constexpr (MODE == MODE_FP64)
                            kuu = kernel_of_dot(A.kernel, A.gamma, A.coef0, A.degree, up.nrm);
                        else if constexpr (MODE == MODE_MIXED)
                            kuu = (double)kernel_of_dot(A.kernel, gammaf, (float)A.coef0, A.degree, (float)up.nrm);
                    }
                    constexpr int RPW = 32 / LPR;
                    const int gl = lane & (LPR - 1);
                    const int gw = lane / LPR;
                    for (int kb = warp * RPW; kb < cnt; kb += kWarps * RPW) {   // warp-uniform
                        const int k = kb + gw;
                        int r = 0;
                        int64_t p0 = 0, p1 = 0;
                        double ft = 0.0;
                        bool cand = false;
                        if (k < cnt) {
                            r = ACT(k);
                            const uint8_t sb = GETST(r);
                            ft = GETF(r);
                            cand = st_low(set_bits(sb)) && kfu < dkey(ft);
                            if (cand) ROWP(r, p0, p1);
                        }
                        Acc su = 0;
                        if (xd) {
                            if constexpr (MODE == MODE_FP64) {
                                const int4 *T4 = reinterpret_cast<const int4 *>(Tn);
                                XdAcc a = xd_zero();
                                for (int64_t p = p0 + gl; p < p1; p += LPR) {
                                    int c;
                                    uint32_t w;
                                    XCW(p, c, w);
                                    const int4 t = T4[c];
                                    xd_add(a, xd_word_m(w), t.x, xd_word_e(w) + t.y);
                                }
                                xd_lane_sum<LPR>(a);
                                su = xd_round(a, xd_unit);
                            }
                        } else {
                            for (int64_t p = p0 + gl; p < p1; p += LPR) {
                                const int c = COL(p);
                                if constexpr (MODE == MODE_BINARY) su += (int)(Tn[c] & 0xff);
                                else if constexpr (MODE == MODE_FP64) su = fma(widen_f32(VAL(p)), Tn[c].x, su);
                                else su = fmaf(VAL(p), Tn[c].x, su);
                            }
#pragma unroll
                            for (int off = LPR / 2; off >= 1; off >>= 1) su += __shfl_xor_sync(0xffffffffu, su, off);
                        }
                        if (cand && gl == 0) {
                            double eta;
                            if constexpr (MODE == MODE_BINARY) {
                                int dist = up.len + (int)(p1 - p0) - 2 * su;
                                eta = etab[dist < 0 ? 0 : dist];
                            } else if (A.kernel == KERNEL_RBF) {
                                double kut;
                                if constexpr (MODE == MODE_FP64) {
                                    const double d2 = up.nrm + NRM(r) - 2.0 * su;
                                    kut = exp_neg_fx(A.gamma * dpos(d2), expfx_s);
                                } else {
                                    const float d2 = (float)up.nrm + NRMF(r) - 2.0f * su;
                                    kut = widen_f32(__expf(-gammaf * fmaxf(d2, 0.f)));
                                }
                                eta = 2.0 - 2.0 * kut;   // K(x,x) = 1
                            } else {
                                double kut, ktt;
                                if constexpr (MODE == MODE_FP64) {
                                    kut = kernel_of_dot(A.kernel, A.gamma, A.coef0, A.degree, (double)su);
                                    ktt = kernel_of_dot(A.kernel, A.gamma, A.coef0, A.degree, NRM(r));
                                } else {
                                    const float c0 = (float)A.coef0;
                                    kut = (double)kernel_of_dot(A.kernel, gammaf, c0, A.degree, (float)su);
                                    ktt = (double)kernel_of_dot(A.kernel, gammaf, c0, A.degree, (float)NRM(r));
                                }
                                eta = __dsub_rn(__dadd_rn(kuu, ktt), __dmul_rn(2.0, kut));
                            }
                            consider(ft, eta, (int)(lo + r), r);
                        }
                    }
                }
                cta_reduce(true, gk, gi, gr, gk, gi, gr, gneg);
                exchange(true);
                if (timed && tid == 0) { uint64_t t = clock64(); ph[7] += t - tp; tp = t; }
                if (sh.res.flag) break;
                low = sh.res.low;
            }
        }
        if (cta == 0 && tid == 0 && iter < A.trace_len) {
            A.trace[2 * iter] = up.i == INT_MAX ? -1 : (A.gmap ? A.gmap[up.i] : up.i);
            A.trace[2 * iter + 1] = low.i == INT_MAX ? -1 : (A.gmap ? A.gmap[low.i] : low.i);
        }
        if (timed && tid == 0) { uint64_t t = clock64(); ph[5] += t - tp; tp = t; }
    }
    cluster.sync();   // no CTA leaves while its shared memory may still be written

    if constexpr (RES) {
        for (int r = tid; r < nseg; r += kThreads) {
            A.f[lo + r] = f_s[r];
            A.alpha[lo + r] = a_s[r];
            A.status[lo + r] = st_s[r];
        }
        for (int k = tid; k < cnt; k += kThreads) A.act[lo + k] = act_s[k];
    }
    if (tid == 0) A.seg_cnt[cta] = cnt;
    if (busy_on && tid == 0) A.cta_cycles[cta] += (int64_t)busy;
    if (cta == 0 && tid == 0) {
        // field by field: ctrl->err may be set concurrently by another CTA
        SmoCtrl *c = A.ctrl;
        c->b_up = up.f;
        c->b_low = low.f;
        c->a_up = up.a;
        c->a_low = low.a;
        c->i_up = up.i == INT_MAX ? -1 : (A.gmap ? A.gmap[up.i] : up.i);
        c->i_low = low.i == INT_MAX ? -1 : (A.gmap ? A.gmap[low.i] : low.i);
        c->iter = iter;
        c->counter = counter;
        c->active = total;
        c->row_visits = row_visits;
        c->exit_reason = exit_reason;
        c->shrink_events = shrink_events;
        for (int k = 0; k < 8; ++k) c->phase_cycles[k] += ph[k];
    }
    if (cta == 0 && tid == kKcThread) {
        A.ctrl->kc_hits += kc_hits;
        A.ctrl->kc_misses += kc_misses;
    }
}

template <int MODE, bool RES, bool SOLO, bool WSS>
void *kernel_for(int lpr)
{
    if constexpr (mode_bits(MODE)) {
        return lpr == 1 ? (void *)smo_persistent_kernel<MODE, 1, RES, SOLO, WSS> : nullptr;
    } else {
        switch (lpr) {
        case 1: return (void *)smo_persistent_kernel<MODE, 1, RES, SOLO, WSS>;
        case 2: return (void *)smo_persistent_kernel<MODE, 2, RES, SOLO, WSS>;
        case 4: return (void *)smo_persistent_kernel<MODE, 4, RES, SOLO, WSS>;
        case 8: return (void *)smo_persistent_kernel<MODE, 8, RES, SOLO, WSS>;
        case 16: return (void *)smo_persistent_kernel<MODE, 16, RES, SOLO, WSS>;
        case 32: return (void *)smo_persistent_kernel<MODE, 32, RES, SOLO, WSS>;
        default: return nullptr;
        }
    }
}

// resident: 0 streamed segments, 1 on-chip segments, 2 on-chip segments in
// one cluster over the whole grid
template <int MODE, bool WSS = false>
void *kernel_pick(int lpr, int resident)
{
    if (resident == 0) return kernel_for<MODE, false, false, WSS>(lpr);
    return resident == 2 ? kernel_for<MODE, true, true, WSS>(lpr) : kernel_for<MODE, true, false, WSS>(lpr);
}

// second-order instantiations, compiled in translation units of their own
void *smo_kernel_wss(int mode, int lpr, int resident);

template <int MODE>
cudaError_t launch_mode(int lpr, const SmoArgs &a, size_t smem, cudaStream_t st, int cs)
{
    const int res = a.resident ? (a.G == cs ? 2 : 1) : 0;
    void *fn = a.wss2 ? smo_kernel_wss(MODE, lpr, res) : kernel_pick<MODE>(lpr, res);
    if (!fn) return cudaErrorInvalidValue;
    if (cs < 1 || a.G % cs != 0 || a.G / cs > 256 || cs > kMaxCluster) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (cs > 8) {
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    SmoArgs args = a;
    void *params[] = {&args};
    // A grid of one cluster is co-scheduled by the hardware; several
    // clusters wait on one another, so that launch is cooperative.
    const bool one_cluster = a.G == cs;
    cudaLaunchAttribute attrs[2];
    attrs[0].id = cudaLaunchAttributeClusterDimension;
    attrs[0].val.clusterDim.x = (unsigned)cs;
    attrs[0].val.clusterDim.y = 1;
    attrs[0].val.clusterDim.z = 1;
    attrs[1].id = cudaLaunchAttributeCooperative;
    attrs[1].val.cooperative = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(a.G);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = attrs;
    cfg.numAttrs = one_cluster ? 1 : 2;
    // all CTAs must be resident at once (they wait on one another)
    int nclusters = 0;
    cudaLaunchConfig_t q = cfg;
    q.attrs = attrs;
    q.numAttrs = 1;
    e = cudaOccupancyMaxActiveClusters(&nclusters, fn, &q);
    if (e != cudaSuccess) return e;
    if (nclusters * cs < a.G) return cudaErrorCooperativeLaunchTooLarge;
    return cudaLaunchKernelExC(&cfg, fn, params);
}

template <int MODE>
int max_clusters(int lpr, int resident, size_t smem, int cs)
{
    void *fn = kernel_pick<MODE>(lpr, resident);
    if (!fn) return 0;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
    if (cs > 8 && cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
        return 0;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = (unsigned)cs;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cudaLaunchConfig_t q = {};
    q.gridDim = dim3(cs);
    q.blockDim = dim3(kThreads);
    q.dynamicSmemBytes = smem;
    q.attrs = &attr;
    q.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, fn, &q) != cudaSuccess) return 0;
    return n;
}

}  // namespace smo
}  // namespace svmgb
