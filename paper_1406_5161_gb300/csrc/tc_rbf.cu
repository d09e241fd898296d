// RBF contraction on the 5th-generation tensor cores (tcgen05, sm_103a):
//
//   out[q] = sum_k coef_k * exp(-gamma * (||z_q||^2 + ||x_k||^2 - 2 <z_q, x_k>))
//
// the inner loop of gradient reconstruction (Algorithm 6: f of the shrunk
// samples from all alpha > 0) and of the decision function (Eq. classi) in
// the mixed-precision mode. The inner products are a dense contraction: query
// rows and support vectors are densified once into BF16 row-major matrices
// (K = columns padded to 64), a CTA keeps a 128-row query tile in shared
// memory and streams 128-row support-vector tiles with TMA (128-byte
// swizzle); one thread issues tcgen05.mma (M = N = 128, K = 16, BF16 inputs,
// FP32 accumulators in tensor memory); the four warps then read the
// 128 x 128 FP32 tile from tensor memory (tcgen05.ld), apply the exp
// epilogue and accumulate coef * K per query row (FP32 within a tile, FP64
// across tiles). Support tiles and accumulators are double-buffered, so the
// load and MMA of the next tile overlap the epilogue. Padding rows carry
// coef = 0.
//
// All waits on mbarriers are bounded; on expiry the CTA records an error,
// waits (bounded) for its own asynchronous work, frees its tensor memory and
// returns, and the host reports SVM_ERR_TIMEOUT.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "svm_internal.cuh"

namespace svmgb {
namespace {

constexpr int kTile = 128;            // rows per query tile and per SV tile (M = N)
constexpr int kKB = 64;               // BF16 elements per 128-byte swizzle row
constexpr int kTcThreads = 320;       // warp 0 loads, warp 1 MMA, warps 2..9 epilogue
constexpr int kMaxKBlocks = 4;        // d_pad <= 256
constexpr uint32_t kTileBytes = kTile * kKB * 2;   // 16 KiB per k-block tile
constexpr long long kWaitLimit = 1ll << 26;        // mbarrier polls before giving up

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// true when the phase with the given parity completed; bounded
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity)
{
    const uint32_t a = smem_u32(bar);
    for (long long i = 0; i < kWaitLimit; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// bulk copy global -> shared counted on an mbarrier (16-byte aligned, size a
// multiple of 16)
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows
// of 128 bytes, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);          // start address
    d |= (uint64_t)1 << 16;                          // leading byte offset (unused here)
    d |= (uint64_t)(1024 >> 4) << 32;                // stride byte offset: 8-row group
    d |= (uint64_t)1 << 46;                          // descriptor version
    d |= (uint64_t)2 << 61;                          // swizzle: 128-byte
    return d;
}

// Instruction descriptor of kind::f16: FP32 accumulate, BF16 A and B, both
// K-major, M = 128, N = 128.
constexpr uint32_t kIdesc = (1u << 4)                  // D format F32
                            | (1u << 7)                // A format BF16
                            | (1u << 10)               // B format BF16
                            | ((uint32_t)(kTile >> 3) << 17)   // N / 8
                            | ((uint32_t)(kTile >> 4) << 24);  // M / 16

struct TcArgs {
    int64_t nq, nsv;
    int kblocks;                 // d_pad / 64
    int stages;                  // support-tile slots in shared memory (2..4)
    const float *zc;             // per query: -gamma * log2(e) * ||z||^2
    const float *xc;             // per SV (padded): -gamma * log2(e) * ||x||^2
    const float *coef;           // per SV (padded): alpha * y (0 on padding)
    float g2;                    // 2 * gamma * log2(e)
    const int32_t *qrow;         // output index per query (row id or position)
    const int8_t *yq;            // subtract yq[qrow] when non-NULL
    double add_scalar;
    double *out;
    int *err;
};

// 2^x on the special-function unit (flush to zero below 2^-126)
// packed pairs of FP32 values (f32x2 arithmetic, sm_100 and later)
__device__ __forceinline__ unsigned long long pack_f32x2(float lo, float hi)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void unpack_f32x2(unsigned long long v, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ unsigned long long add_f32x2(unsigned long long a, unsigned long long b)
{
    unsigned long long r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ unsigned long long fma_f32x2(unsigned long long a, unsigned long long b,
                                                       unsigned long long c)
{
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// One CTA: a 128-row query tile against all support-vector tiles, with the
// roles split by warp and handed over by mbarriers only (no CTA-wide barrier
// inside the tile loop):
//   warp 0 (one thread)  TMA loads of the support tiles and their constants
//                        into a ring of `stages` shared-memory slots;
//   warp 1 (one thread)  tcgen05.mma of each tile into one of two 128-column
//                        tensor-memory accumulators;
//   warps 2..9           the epilogue: each reads its 32-lane quadrant
//                        (warp % 4) and half of the columns of an accumulator
//                        with tcgen05.ld, evaluates coef * 2^(...) and sums.
// full[s]  : the tile in slot s has landed (TMA transaction bytes);
// empty[s] : slot s is free again (the MMA's commit + one arrival per
//            epilogue warp, which also read the slot's constants);
// accf[b]  : accumulator b holds a finished tile (MMA commit);
// acce[b]  : the epilogue has read accumulator b (one arrival per warp).
// Tile t uses slot t % stages (round t / stages) and accumulator t & 1 (use
// t >> 1); the k-th completion of a barrier has parity k & 1.
constexpr int kEpiWarps = 8;
constexpr int kMaxStages = 4;

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait that also gives up once another role has failed. The thread
// sleeps in the barrier (suspend-time hint) until the phase completes or the
// hint runs out, so waiting warps take no issue slots from the epilogue; the
// whole wait is bounded by kWaitNs of the global timer.
constexpr uint64_t kWaitNs = 5ull * 1000 * 1000 * 1000;
__device__ __forceinline__ bool mbar_wait_or_fail(uint64_t *bar, uint32_t parity, const volatile int *fail)
{
    const uint32_t a = smem_u32(bar);
    uint64_t t0 = 0;
    for (;;) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(a), "r"(parity), "r"(20000u)
            : "memory");
        if (ok) return true;
        if (*fail) return false;
        const uint64_t now = global_ns();
        if (t0 == 0) t0 = now;
        else if (now - t0 > kWaitNs) return false;
    }
}

__global__ void __launch_bounds__(kTcThreads) tc_rbf_kernel(const __grid_constant__ CUtensorMap mapZ,
                                                            const __grid_constant__ CUtensorMap mapX,
                                                            TcArgs a)
{
    extern __shared__ __align__(1024) unsigned char dsm_raw[];
    // 1024-byte alignment for the swizzled tiles
    unsigned char *dsm = reinterpret_cast<unsigned char *>(((uintptr_t)dsm_raw + 1023) & ~(uintptr_t)1023);
    const int S = a.stages;
    const size_t tile_all = (size_t)a.kblocks * kTileBytes;   // one tile, all k-blocks
    unsigned char *tileA = dsm;                               // the query tile
    unsigned char *tileB = dsm + tile_all;                    // [S][kblocks][16 KiB]
    __shared__ __align__(8) uint64_t bar_q, bar_full[kMaxStages], bar_empty[kMaxStages], bar_accf[2],
        bar_acce[2], bar_drain;
    __shared__ uint32_t tmem_base;
    __shared__ __align__(16) float s_xc[kMaxStages][kTile], s_coef[kMaxStages][kTile];
    __shared__ double s_acc[kTile];   // the second column half's row sums
    __shared__ int s_fail;
    const volatile int *fail = &s_fail;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t q0 = (int64_t)blockIdx.x * kTile;
    if (tid == 0) {
        mbar_init(&bar_q, 1);
        for (int k = 0; k < kMaxStages; ++k) {
            mbar_init(&bar_full[k], 1);
            mbar_init(&bar_empty[k], 1 + kEpiWarps);
        }
        for (int k = 0; k < 2; ++k) {
            mbar_init(&bar_accf[k], 1);
            mbar_init(&bar_acce[k], kEpiWarps);
        }
        mbar_init(&bar_drain, 1);
        s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(&tmem_base)), "r"(2 * kTile) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    const int64_t ntiles = (a.nsv + kTile - 1) / kTile;

    bool ok = true;
    int64_t issued = 0;         // producer: support tiles whose loads were issued
    bool q_issued = false;
    const int quad = warp & 3, half = (warp - 2) >> 2;    // epilogue warps
    const int my_row = quad * 32 + lane;                  // TMEM lane = query row in tile
    double acc = 0.0;

    if (warp == 0) {
        // ---- producer
        if (lane == 0) {
            mbar_expect_tx(&bar_q, (uint32_t)tile_all);
            for (int kb = 0; kb < a.kblocks; ++kb)
                tma_load_2d(tileA + (size_t)kb * kTileBytes, &mapZ, kb * kKB, (int)q0, &bar_q);
            q_issued = true;
            for (int64_t t = 0; t < ntiles; ++t) {
                const int sl = (int)(t % S);
                const int64_t r = t / S;
                if (r >= 1 && !mbar_wait_or_fail(&bar_empty[sl], (uint32_t)((r - 1) & 1), fail)) {
                    ok = false;
                    break;
                }
                // the slot's last readers included the epilogue's generic loads
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                unsigned char *tb = tileB + (size_t)sl * tile_all;
                mbar_expect_tx(&bar_full[sl], (uint32_t)tile_all + 2 * kTile * 4);
                for (int kb = 0; kb < a.kblocks; ++kb)
                    tma_load_2d(tb + (size_t)kb * kTileBytes, &mapX, kb * kKB, (int)(t * kTile), &bar_full[sl]);
                bulk_load(s_xc[sl], a.xc + t * kTile, kTile * 4, &bar_full[sl]);
                bulk_load(s_coef[sl], a.coef + t * kTile, kTile * 4, &bar_full[sl]);
                issued = t + 1;
            }
        }
    } else if (warp == 1) {
        // ---- MMA issue: D[b] = Z_tile * X_tile^T over all K
        if (lane == 0) {
            ok = mbar_wait_or_fail(&bar_q, 0, fail);
            for (int64_t t = 0; ok && t < ntiles; ++t) {
                const int sl = (int)(t % S), b = (int)(t & 1);
                const int64_t r = t / S, u = t >> 1;
                if (!mbar_wait_or_fail(&bar_full[sl], (uint32_t)(r & 1), fail) ||
                    (u >= 1 && !mbar_wait_or_fail(&bar_acce[b], (uint32_t)((u - 1) & 1), fail))) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const unsigned char *tb = tileB + (size_t)sl * tile_all;
                const uint32_t dcol = tmem + (uint32_t)(b * kTile);
                for (int kb = 0; kb < a.kblocks; ++kb) {
                    const uint32_t sa = smem_u32(tileA + (size_t)kb * kTileBytes);
                    const uint32_t sb = smem_u32(tb + (size_t)kb * kTileBytes);
#pragma unroll
                    for (int ks = 0; ks < kKB / 16; ++ks) {
                        const uint64_t da = smem_desc_sw128(sa + ks * 32);
                        const uint64_t db = smem_desc_sw128(sb + ks * 32);
                        const uint32_t accum = (kb | ks) ? 1u : 0u;
                        asm volatile(
                            "{\n\t.reg .pred p;\n\t"
                            "setp.ne.b32 p, %4, 0;\n\t"
                            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                            ::"r"(dcol), "l"(da), "l"(db), "r"(kIdesc), "r"(accum)
                            : "memory");
                    }
                }
                // both fire when these MMAs are done: the accumulator is
                // ready, and the MMA no longer reads the slot
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                             ::"r"(smem_u32(&bar_accf[b])) : "memory");
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                             ::"r"(smem_u32(&bar_empty[sl])) : "memory");
            }
        }
    } else {
        // ---- epilogue
        const int64_t q = q0 + my_row;
        const float zc = (q < a.nq) ? a.zc[q] : 0.f;
        const unsigned long long zc2 = pack_f32x2(zc, zc), g2v = pack_f32x2(a.g2, a.g2);
        // The row's scaled norm factors out of the sum:
        //   sum_j c_j 2^min(g2 dot_j + xc_j + zc, 0)
        //     = 2^zc sum_j c_j 2^min(g2 dot_j + xc_j, -zc),
        // one addition less per pair; 2^zc is applied once per tile. A warp
        // with a row whose 2^-zc would leave FP32 (-zc > 120) keeps the
        // per-pair form.
        const float nzc = -zc;
        const bool factored = !__any_sync(0xffffffffu, nzc > 120.f);
        const double row_scale = factored ? exp2((double)zc) : 1.0;
        for (int64_t t = 0; t < ntiles; ++t) {
            const int sl = (int)(t % S), b = (int)(t & 1);
            const int64_t r = t / S, u = t >> 1;
            const bool w_ok = mbar_wait_or_fail(&bar_accf[b], (uint32_t)(u & 1), fail) &&
                              mbar_wait_or_fail(&bar_full[sl], (uint32_t)(r & 1), fail);
            if (!__all_sync(0xffffffffu, w_ok)) {
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            // (columns j, j + 1) partial sums, two chains
            unsigned long long partA = pack_f32x2(0.f, 0.f), partB = partA;
#pragma unroll 1
            for (int c0 = half * (kTile / 2); c0 < (half + 1) * (kTile / 2); c0 += 32) {
                uint32_t rr[32];
                const uint32_t addr = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(b * kTile + c0);
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                    "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                    "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                    : "=r"(rr[0]), "=r"(rr[1]), "=r"(rr[2]), "=r"(rr[3]), "=r"(rr[4]), "=r"(rr[5]), "=r"(rr[6]),
                      "=r"(rr[7]), "=r"(rr[8]), "=r"(rr[9]), "=r"(rr[10]), "=r"(rr[11]), "=r"(rr[12]),
                      "=r"(rr[13]), "=r"(rr[14]), "=r"(rr[15]), "=r"(rr[16]), "=r"(rr[17]), "=r"(rr[18]),
                      "=r"(rr[19]), "=r"(rr[20]), "=r"(rr[21]), "=r"(rr[22]), "=r"(rr[23]), "=r"(rr[24]),
                      "=r"(rr[25]), "=r"(rr[26]), "=r"(rr[27]), "=r"(rr[28]), "=r"(rr[29]), "=r"(rr[30]),
                      "=r"(rr[31])
                    : "r"(addr)
                    : "memory");
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                // the FP32 arithmetic runs on packed column pairs (f32x2),
                // the same IEEE result in each lane as the scalar form
                const float4 *xs = reinterpret_cast<const float4 *>(&s_xc[sl][c0]);
                const float4 *cs = reinterpret_cast<const float4 *>(&s_coef[sl][c0]);
                if (factored) {
#pragma unroll
                    for (int v = 0; v < 8; ++v) {
                        const float4 x4 = xs[v], c4 = cs[v];   // the same address in every lane
                        const int j = 4 * v;
                        float e0, e1, e2, e3;
                        unpack_f32x2(fma_f32x2(pack_f32x2(__uint_as_float(rr[j]), __uint_as_float(rr[j + 1])), g2v,
                                               pack_f32x2(x4.x, x4.y)), e0, e1);
                        unpack_f32x2(fma_f32x2(pack_f32x2(__uint_as_float(rr[j + 2]), __uint_as_float(rr[j + 3])),
                                               g2v, pack_f32x2(x4.z, x4.w)), e2, e3);
                        const unsigned long long k01 = pack_f32x2(ex2_approx(fminf(e0, nzc)), ex2_approx(fminf(e1, nzc)));
                        const unsigned long long k23 = pack_f32x2(ex2_approx(fminf(e2, nzc)), ex2_approx(fminf(e3, nzc)));
                        partA = fma_f32x2(pack_f32x2(c4.x, c4.y), k01, partA);
                        partB = fma_f32x2(pack_f32x2(c4.z, c4.w), k23, partB);
                    }
                } else {
#pragma unroll
                    for (int v = 0; v < 8; ++v) {
                        const float4 x4 = xs[v], c4 = cs[v];
                        const int j = 4 * v;
                        float e0, e1, e2, e3;
                        unpack_f32x2(fma_f32x2(pack_f32x2(__uint_as_float(rr[j]), __uint_as_float(rr[j + 1])), g2v,
                                               add_f32x2(pack_f32x2(x4.x, x4.y), zc2)), e0, e1);
                        unpack_f32x2(fma_f32x2(pack_f32x2(__uint_as_float(rr[j + 2]), __uint_as_float(rr[j + 3])),
                                               g2v, add_f32x2(pack_f32x2(x4.z, x4.w), zc2)), e2, e3);
                        const unsigned long long k01 = pack_f32x2(ex2_approx(fminf(e0, 0.f)), ex2_approx(fminf(e1, 0.f)));
                        const unsigned long long k23 = pack_f32x2(ex2_approx(fminf(e2, 0.f)), ex2_approx(fminf(e3, 0.f)));
                        partA = fma_f32x2(pack_f32x2(c4.x, c4.y), k01, partA);
                        partB = fma_f32x2(pack_f32x2(c4.z, c4.w), k23, partB);
                    }
                }
            }
            float pa0, pa1, pb0, pb1;
            unpack_f32x2(partA, pa0, pa1);
            unpack_f32x2(partB, pb0, pb1);
            acc += (double)((pa0 + pa1) + (pb0 + pb1)) * row_scale;
            // this warp is done with accumulator b and with slot sl
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&bar_acce[b]);
                mbar_arrive(&bar_empty[sl]);
            }
        }
    }
    if (!ok && lane == 0) {
        s_fail = 1;
        atomicExch(a.err, 1);
    }
    __syncthreads();
    if (s_fail) {
        // let this CTA's outstanding asynchronous work finish (bounded)
        // before its shared and tensor memory are released
        if (warp == 1 && lane == 0) {
            // a commit tracks every earlier MMA of this thread
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         ::"r"(smem_u32(&bar_drain)) : "memory");
            (void)mbar_wait(&bar_drain, 0);
        }
        if (warp == 0 && lane == 0) {
            // loads in flight: at most the last `stages` tiles, one per slot
            for (int64_t t = issued > S ? issued - S : 0; t < issued; ++t)
                (void)mbar_wait(&bar_full[t % S], (uint32_t)((t / S) & 1));
            if (q_issued) (void)mbar_wait(&bar_q, 0);
        }
    } else {
        // the two column halves of a row meet in shared memory (fixed order)
        if (warp >= 2 && half == 1) s_acc[my_row] = acc;
        __syncthreads();
        if (warp >= 2 && half == 0) {
            const int64_t q = q0 + my_row;
            if (q < a.nq) {
                const int32_t row = a.qrow[q];
                double v = (acc + s_acc[my_row]) + a.add_scalar;
                if (a.yq) v -= (double)a.yq[row];
                a.out[row] = v;
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kTile)
                     : "memory");
    }
}

// ------------------------------------------------------------- preparation

// Dense BF16 rows (row-major, ld = d_pad) from CSR rows (list or all) and the
// scaled norms used by the epilogue; padding rows are zero.
__global__ void k_densify(int64_t nrows, int64_t nrows_pad, int d_pad, const int32_t *list,
                          const int64_t *indptr, const int32_t *indices, const float *vmix,
                          const float *normf, float nscale, __nv_bfloat16 *dense, float *cnorm,
                          const double *coef_in, float *coef_out, int32_t *outrow, int out_by_row)
{
    const int64_t r = blockIdx.x;
    if (r >= nrows_pad) return;
    __nv_bfloat16 *dst = dense + (size_t)r * d_pad;
    for (int c = threadIdx.x; c < d_pad; c += blockDim.x) dst[c] = __float2bfloat16_rn(0.f);
    __syncthreads();
    if (r < nrows) {
        const int64_t row = list ? list[r] : r;
        for (int64_t p = indptr[row] + threadIdx.x; p < indptr[row + 1]; p += blockDim.x)
            dst[indices[p]] = __float2bfloat16_rn(vmix[p]);
        if (threadIdx.x == 0) {
            cnorm[r] = nscale * normf[row];
            if (coef_out) coef_out[r] = (float)coef_in[r];
            if (outrow) outrow[r] = out_by_row ? (int32_t)row : (int32_t)r;
        }
    } else if (threadIdx.x == 0) {
        cnorm[r] = 0.f;
        if (coef_out) coef_out[r] = 0.f;
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

bool make_map(CUtensorMap *m, const void *base, int64_t rows, int d_pad)
{
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)d_pad, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)d_pad * 2};
    cuuint32_t box[2] = {(cuuint32_t)kKB, (cuuint32_t)kTile};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

}  // namespace

bool tc_rbf_supported(int d) { return d >= 1 && d <= kMaxKBlocks * kKB && encode_fn() != nullptr; }

size_t tc_rbf_workspace_bytes(int64_t nq, int64_t nsv, int d)
{
    const int d_pad = ((d + kKB - 1) / kKB) * kKB;
    const int64_t nq_pad = (nq + kTile - 1) / kTile * kTile;
    const int64_t ns_pad = (nsv + kTile - 1) / kTile * kTile;
    size_t b = 0;
    auto add = [&](size_t x) { b += (x + 255) & ~(size_t)255; };
    add((size_t)nq_pad * d_pad * 2);
    add((size_t)ns_pad * d_pad * 2);
    add((size_t)nq_pad * 4);   // zc
    add((size_t)ns_pad * 4);   // xc
    add((size_t)ns_pad * 4);   // coef
    add((size_t)nq_pad * 4);   // qrow
    add(256);                  // err
    return b;
}

// Same contract as launch_rbf_contract (MODE_MIXED inputs: vmix values and
// FP32 norms), on the tensor cores. `ws` must hold tc_rbf_workspace_bytes.
cudaError_t launch_rbf_contract_tc(const RbfContract &c, void *ws, int *err_host, cudaStream_t st)
{
    *err_host = 0;
    if (c.nq <= 0) return cudaSuccess;
    const int d_pad = ((c.d + kKB - 1) / kKB) * kKB;
    const int kblocks = d_pad / kKB;
    if (kblocks > kMaxKBlocks) return cudaErrorInvalidValue;
    const int64_t nq_pad = (c.nq + kTile - 1) / kTile * kTile;
    const int64_t ns = c.nsv > 0 ? c.nsv : 1;
    const int64_t ns_pad = (ns + kTile - 1) / kTile * kTile;
    unsigned char *p = static_cast<unsigned char *>(ws);
    auto take = [&](size_t x) {
        unsigned char *r = p;
        p += (x + 255) & ~(size_t)255;
        return r;
    };
    auto *Zd = reinterpret_cast<__nv_bfloat16 *>(take((size_t)nq_pad * d_pad * 2));
    auto *Xd = reinterpret_cast<__nv_bfloat16 *>(take((size_t)ns_pad * d_pad * 2));
    auto *zc = reinterpret_cast<float *>(take((size_t)nq_pad * 4));
    auto *xc = reinterpret_cast<float *>(take((size_t)ns_pad * 4));
    auto *coef = reinterpret_cast<float *>(take((size_t)ns_pad * 4));
    auto *qrow = reinterpret_cast<int32_t *>(take((size_t)nq_pad * 4));
    auto *err = reinterpret_cast<int *>(take(256));
    const float L2E = 1.4426950408889634f;
    const float nscale = (float)(-c.gamma) * L2E;
    cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    k_densify<<<(unsigned)nq_pad, 64, 0, st>>>(c.nq, nq_pad, d_pad, c.q, c.z_indptr, c.z_indices, c.z_values,
                                               c.z_normf, nscale, Zd, zc, nullptr, nullptr, qrow, c.out_by_row);
    k_densify<<<(unsigned)ns_pad, 64, 0, st>>>(c.nsv, ns_pad, d_pad, c.sv, c.x_indptr, c.x_indices, c.x_values,
                                               c.x_normf, nscale, Xd, xc, c.coef, coef, nullptr, 0);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    CUtensorMap mz, mx;
    if (!make_map(&mz, Zd, nq_pad, d_pad) || !make_map(&mx, Xd, ns_pad, d_pad)) return cudaErrorInvalidValue;
    TcArgs a;
    a.nq = c.nq;
    a.nsv = c.nsv;
    a.kblocks = kblocks;
    a.zc = zc;
    a.xc = xc;
    a.coef = coef;
    a.g2 = 2.0f * (float)c.gamma * L2E;
    a.qrow = qrow;
    a.yq = c.yq;
    a.add_scalar = c.add_scalar;
    a.out = c.out;
    a.err = err;
    // query tile + a ring of support tiles: 4 slots at d <= 64, else 2; at
    // least 80 KiB so that at most 2 CTAs share an SM: their 2 x 256
    // tensor-memory columns then fit the SM's 512 without waiting
    a.stages = kblocks == 1 ? 4 : 2;
    const size_t smem = std::max<size_t>((size_t)(1 + a.stages) * kblocks * kTileBytes + 1024, 80 * 1024);
    e = cudaFuncSetAttribute(tc_rbf_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (c.nsv > 0) {
        tc_rbf_kernel<<<(unsigned)(nq_pad / kTile), kTcThreads, smem, st>>>(mz, mx, a);
    } else {
        // no support vectors: every sum is zero
        return cudaErrorInvalidValue;
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(err_host, err, sizeof(int), cudaMemcpyDeviceToHost, st);
    return e;
}


// SFU exp2 rate (microbenchmark for the contraction's roofline): every thread
// runs 8 independent chains of ex2.approx, the instruction of the epilogue.
__global__ void k_sfu_ex2(int iters, float seed, float *sink)
{
    float a[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = seed * (float)(j + 1) * 1e-3f - (float)(threadIdx.x & 7) * 1e-4f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            float r;
            asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a[j]));
            a[j] = r * -0.5f;   // stays in (-1, 1): no overflow, no denormals
        }
    }
    float acc = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) acc += a[j];
    if (acc == 12345.f) sink[blockIdx.x] = acc;   // keeps the loop alive
}

cudaError_t measure_sfu_ex2(double *ops_per_s, cudaStream_t st)
{
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int blocks = sms * 8, threads = 256, iters = 4096;
    float *sink = nullptr;
    if ((e = cudaMallocAsync(&sink, sizeof(float) * blocks, st)) != cudaSuccess) return e;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k_sfu_ex2<<<blocks, threads, 0, st>>>(iters / 8, 0.5f, sink);   // warm-up
    cudaEventRecord(e0, st);
    k_sfu_ex2<<<blocks, threads, 0, st>>>(iters, 0.5f, sink);
    cudaEventRecord(e1, st);
    e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFreeAsync(sink, st);
    if (e == cudaSuccess) *ops_per_s = (double)blocks * threads * iters * 8 / (ms * 1e-3);
    return e;
}

}  // namespace svmgb
