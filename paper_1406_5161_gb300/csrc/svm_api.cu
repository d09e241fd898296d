// C ABI of the GB300 SVM library: ingest, the SMO driver (Algorithms 1, 4,
// 5 and 6 of arXiv:1406.5161), the decision function and utilities.
//
// Host code here only orchestrates: every arithmetic step of training and
// prediction runs in the library's CUDA kernels. The host reads a small
// control block between phases (after each persistent launch) to apply the
// phase logic of Algorithm 5.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <new>
#include <mutex>
#include <thread>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "svm_internal.cuh"

using namespace svmgb;

namespace {

thread_local std::string g_err;
std::atomic<long long> g_launches{0};

void set_err(const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
}

struct Fail {
    int code;
};

#define CK(call)                                                                         \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess) {                                                         \
            set_err("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__,   \
                    __LINE__);                                                           \
            throw Fail{e_ == cudaErrorMemoryAllocation ? SVM_ERR_OOM : SVM_ERR_CUDA};   \
        }                                                                                \
    } while (0)

#define CK_NOTHROW(call) (void)(call)

#define ARG_FAIL(...)                 \
    do {                              \
        set_err(__VA_ARGS__);         \
        throw Fail{SVM_ERR_ARG};      \
    } while (0)

// Stream-ordered device allocations released when the scope ends.
struct Arena {
    cudaStream_t st;
    std::vector<void *> ptrs;
    explicit Arena(cudaStream_t s) : st(s) {}
    template <class T>
    T *alloc(size_t count)
    {
        void *p = nullptr;
        if (count == 0) count = 1;
        CK(cudaMallocAsync(&p, count * sizeof(T), st));
        ptrs.push_back(p);
        return static_cast<T *>(p);
    }
    ~Arena()
    {
        for (void *p : ptrs) cudaFreeAsync(p, st);
        cudaStreamSynchronize(st);
    }
};

// --------------------------------------------------------------- kernels

struct IngestInfo {
    int bad_indptr;
    int bad_index;
    int bad_y;
    int nonfinite;
    int not_binary;
    int pad;
    unsigned long long npos;
    int maxnnz;
    int pad2;
    // biased exponents of the nonzero values: the largest, 255 - the
    // smallest, and whether a subnormal value occurs (exact inner products)
    int bmax;
    int nbmin;
    int subnormal;
    int pad3;
};

// Validates the CSR structure and labels; detects binary (all 1.0) values;
// the longest row and the exponent range of the values (one atomic per warp).
__global__ void k_validate(int64_t n, int64_t d, const int64_t *indptr, const int32_t *indices,
                           const float *values, const int8_t *y, IngestInfo *info)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int len = 0, bmax = 0, nbmin = 0, sub = 0;
    if (i < n) {
        const int64_t p0 = indptr[i], p1 = indptr[i + 1];
        if (p1 < p0 || (i == 0 && p0 != 0)) {
            atomicOr(&info->bad_indptr, 1);
        } else {
            int prev = -1;
            bool nb = false, nf = false, bi = false;
            for (int64_t p = p0; p < p1; ++p) {
                int c = indices[p];
                if (c <= prev || c >= d) bi = true;
                prev = c;
                if (values) {
                    const float v = values[p];
                    if (!isfinite(v)) nf = true;
                    if (v != 1.0f) nb = true;
                    const uint32_t u = __float_as_uint(v);
                    const int b = (int)((u >> 23) & 0xffu);
                    if (b != 0) {
                        bmax = max(bmax, b);
                        nbmin = max(nbmin, 255 - b);
                    } else if (u & 0x007fffffu) {
                        sub = 1;
                    }
                }
            }
            if (bi) atomicOr(&info->bad_index, 1);
            if (nf) atomicOr(&info->nonfinite, 1);
            if (nb) atomicOr(&info->not_binary, 1);
            len = (int)(p1 - p0);
            if (y) {
                int8_t v = y[i];
                if (v != 1 && v != -1) atomicOr(&info->bad_y, 1);
                if (v == 1) atomicAdd(&info->npos, 1ull);
            }
        }
    }
    len = __reduce_max_sync(0xffffffffu, len);
    bmax = __reduce_max_sync(0xffffffffu, bmax);
    nbmin = __reduce_max_sync(0xffffffffu, nbmin);
    sub = __reduce_or_sync(0xffffffffu, sub);
    if ((threadIdx.x & 31) == 0) {
        if (len) atomicMax(&info->maxnnz, len);
        if (bmax) atomicMax(&info->bmax, bmax);
        if (nbmin) atomicMax(&info->nbmin, nbmin);
        if (sub) atomicOr(&info->subnormal, 1);
    }
}

// Mixed rows for the row pass: each stored entry as one word, the column
// (< 2^16) in bits 0-15 and the BF16-rounded value's bits in 16-31 (its
// FP32 copy has zero low half, so nothing is lost).
__global__ void k_pack_ew(int64_t nnz, const int32_t *indices, const float *vmix, uint32_t *ew)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < nnz) ew[p] = (__float_as_uint(vmix[p]) & 0xffff0000u) | (uint32_t)indices[p];
}

// FP64 rows with exact inner products: each stored entry as its column
// (< 2^16) in bits 0-15 and the (m, b - t) word of its value in 16-47.
__global__ void k_pack_ew64(int64_t nnz, const int32_t *indices, const float *values, int tmin, uint64_t *ew64)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < nnz) ew64[p] = ((uint64_t)xd_word(__float_as_uint(values[p]), tmin) << 16) | (uint32_t)indices[p];
}

// The exact-inner-product format of one matrix from its validation record
// (values NULL: every value is 1.0); host and device compute the same.
__host__ __device__ XdFormat xd_of_info(const IngestInfo &h, const float *values)
{
    const int bmax = values ? h.bmax : 127, bmin = values ? 255 - h.nbmin : 127;
    return xd_format(bmax, bmin, h.maxnnz, values && h.subnormal != 0);
}

// ||x_i||^2 in FP64: exact and rounded once when the matrix's format allows
// (the inner product of the row with itself, as the row passes compute it),
// else summed in row order; and the BF16-rounded copy with its FP32 norm.
// info: the matrix's validation record, written by k_validate before.
__global__ void k_norms(int64_t n, const int64_t *indptr, const float *values, double *norm,
                        float *vmix, float *normf, const IngestInfo *info)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const XdFormat xd = xd_of_info(*info, values);
    int64_t p0 = indptr[i], p1 = indptr[i + 1];
    double s = 0.0;
    XdAcc a = xd_zero();
    float sf = 0.f;
    for (int64_t p = p0; p < p1; ++p) {
        float v = values ? values[p] : 1.0f;
        if (xd.on) {
            const uint32_t u = __float_as_uint(v);
            const int32_t m = xd_mant(u);
            xd_add(a, m, m, 2 * xd_exp(u, xd.tmin) + xd.bias);
        } else {
            s += (double)v * (double)v;
        }
        if (vmix) {
            float r = __bfloat162float(__float2bfloat16_rn(v));
            vmix[p] = r;
            sf = fmaf(r, r, sf);
        }
    }
    if (norm) norm[i] = xd.on ? xd_round(a, xd.unit) : s;
    if (normf) normf[i] = sf;
}

// Tables over the integer squared distances k of binary rows (3 len
// doubles): exp(-gamma * k); the correctly rounded reciprocal of
// eta = 2 - 2 exp(-gamma k) used by the pair step (0 where eta <= 1e-12);
// eta itself.
__global__ void k_ktab(double gamma, int len, double *ktab)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < len) {
        const double kv = exp(-gamma * (double)k);
        const double eta = 2.0 - 2.0 * kv;
        ktab[k] = kv;
        ktab[len + k] = eta > 1e-12 ? 1.0 / eta : 0.0;
        ktab[2 * len + k] = eta;
    }
}

// alpha = 0, f = -y (Algorithm 1 initialisation), index sets from y.
__global__ void k_init(int64_t n, const int8_t *y, double *alpha, double *f, uint8_t *status)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int8_t yi = y[i];
    alpha[i] = 0.0;
    f[i] = -(double)yi;
    status[i] = (uint8_t)(st_of(yi, 0.0, 1.0) | (yi > 0 ? 0x80 : 0));
}

// Warm start: the given multipliers and their index sets (Eq. setinfo).
__global__ void k_init_warm(int64_t n, double C, const int8_t *y, const double *alpha0, double *alpha,
                            uint8_t *status)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int8_t yi = y[i];
    const double a = alpha0[i];
    alpha[i] = a;
    status[i] = (uint8_t)(st_of(yi, a, C) | (yi > 0 ? 0x80 : 0));
}

// Active lists back to all samples: segment s holds local indices 0..size-1.
__global__ void k_reset_active(int64_t n, int G, int32_t *act, int32_t *seg_cnt)
{
    const int s = blockIdx.x;
    const int64_t lo = seg_lo(n, G, s);
    const int m = (int)(seg_lo(n, G, s + 1) - lo);
    for (int r = threadIdx.x; r < m; r += blockDim.x) act[lo + r] = r;
    if (threadIdx.x == 0) seg_cnt[s] = m;
}

// mark[i] = 1 for samples in an active list.
__global__ void k_mark_active(int64_t n, int G, const int32_t *act, const int32_t *seg_cnt,
                              uint8_t *mark)
{
    const int s = blockIdx.x;
    const int64_t lo = seg_lo(n, G, s);
    for (int k = threadIdx.x; k < seg_cnt[s]; k += blockDim.x) mark[lo + act[lo + k]] = 1;
}

// Incremental reconstruction. For the m rows gathered into a re-layout level
// (idx: their rows in the caller's problem, a0: their alpha at the gather):
// the change of alpha since the gather at each such row (dalpha, marked in
// dmark when not zero) and a mark of the gathered rows.
__global__ void k_inc_delta(int64_t m, const int32_t *idx, const double *a0, const double *alpha,
                            double *dalpha, uint8_t *dmark, uint8_t *gathered)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= m) return;
    const int i = idx[k];
    const double d = alpha[i] - a0[k];
    dalpha[i] = d;
    dmark[i] = d != 0.0;
    gathered[i] = 1;
}

// Query marks of the two reconstructions (a row is a query where its mark is
// 0): q1 the rows shrunk before the gather, q2 the gathered rows shrunk after.
__global__ void k_inc_marks(int64_t n, const uint8_t *active, const uint8_t *gathered, uint8_t *q1,
                            uint8_t *q2)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    q1[i] = (uint8_t)(active[i] | gathered[i]);
    q2[i] = (uint8_t)!(gathered[i] && !active[i]);
}

// stored entries per segment
__global__ void k_seg_nnz(int64_t n, int G, const int64_t *indptr, int64_t *out)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < G) out[s] = indptr[seg_lo(n, G, s + 1)] - indptr[seg_lo(n, G, s)];
}

__global__ void k_dense_bf16(int64_t n, int d, int d_pad, const int64_t *indptr, const int32_t *indices,
                             const float *vmix, __nv_bfloat16 *out);
__global__ void k_iota(int64_t n, int32_t *out);

// ---- active-set re-layout: the active rows of a problem gathered into a
//      smaller problem (rows kept in increasing index order, so the
//      lowest-index tie-break is unchanged), and the solver state scattered
//      back when the smaller problem's launch ends

// stored entries of the selected rows, per chunk of kChunkRows rows
constexpr int kChunkRows = 4096;
// largest FP64-mode problem (rows, non-binary input) solved by one 16-CTA cluster
constexpr int64_t kFp64OneClusterRows = 8192;
// smallest FP64-mode problem that takes one CTA per SM with the flat exchange
// even when its segments fit in shared memory
constexpr int64_t kFp64FlatRows = 200000;
__global__ void k_sub_len_sums(int64_t m, const int32_t *idx, const int64_t *indptr, int64_t *sums)
{
    __shared__ unsigned long long s;
    if (threadIdx.x == 0) s = 0;
    __syncthreads();
    const int64_t b0 = (int64_t)blockIdx.x * kChunkRows;
    unsigned long long c = 0;
    for (int64_t j = b0 + threadIdx.x; j < m && j < b0 + kChunkRows; j += blockDim.x)
        c += (unsigned long long)(indptr[idx[j] + 1] - indptr[idx[j]]);
    atomicAdd(&s, c);
    __syncthreads();
    if (threadIdx.x == 0) sums[blockIdx.x] = (int64_t)s;
}

__global__ void k_scan64(const int64_t *sums, int nb, int64_t *offs, int64_t *total)
{
    if (threadIdx.x != 0) return;
    int64_t acc = 0;
    for (int b = 0; b < nb; ++b) {
        offs[b] = acc;
        acc += sums[b];
    }
    *total = acc;
}

// row pointers of the selected rows: per chunk, an ordered block scan of
// their lengths (256 threads)
__global__ void k_sub_indptr(int64_t m, const int32_t *idx, const int64_t *indptr, const int64_t *offs,
                             int64_t *sub_indptr)
{
    __shared__ int64_t wsum[8];
    __shared__ int64_t base;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x == 0) base = offs[blockIdx.x];
    __syncthreads();
    const int64_t b0 = (int64_t)blockIdx.x * kChunkRows;
    for (int64_t s0 = b0; s0 < m && s0 < b0 + kChunkRows; s0 += 256) {
        const int64_t j = s0 + threadIdx.x;
        const int64_t len = (j < m && j < b0 + kChunkRows) ? indptr[idx[j] + 1] - indptr[idx[j]] : 0;
        int64_t incl = len;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int64_t o = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += o;
        }
        if (lane == 31) wsum[w] = incl;
        __syncthreads();
        int64_t pre = base + incl - len;
        int64_t tot = 0;
        for (int k = 0; k < 8; ++k) {
            if (k < w) pre += wsum[k];
            tot += wsum[k];
        }
        if (j < m && j < b0 + kChunkRows) sub_indptr[j] = pre;
        __syncthreads();
        if (threadIdx.x == 0) base += tot;
        __syncthreads();
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) sub_indptr[m] = base;
}

// the selected rows' entries (one warp per row) and per-row data
struct SubRowsArgs {
    int64_t m;
    const int32_t *idx;          // selected rows of the parent problem
    const int32_t *pmap;         // parent index -> caller index (NULL: identity)
    const int64_t *indptr;
    const int32_t *indices;
    const float *values, *vmix, *normf;
    const double *norm, *alpha, *f;
    const int8_t *y;
    const uint8_t *status;
    const uint32_t *bits;
    int bit_words;
    const int64_t *sub_indptr;
    int32_t *sub_indices;
    float *sub_values, *sub_vmix, *sub_normf;
    double *sub_norm, *sub_alpha, *sub_f;
    int8_t *sub_y;
    uint8_t *sub_status;
    uint32_t *sub_bits;
    const uint32_t *ew;          // mixed rows one word per entry, or NULL
    uint32_t *sub_ew;
    const uint64_t *ew64;        // FP64 rows, packed entries, or NULL
    uint64_t *sub_ew64;
    int32_t *sub_gmap;
    const __nv_bfloat16 *dmat;   // dense BF16 rows (tensor-core row tiles), or NULL
    __nv_bfloat16 *sub_dmat;
    int d_pad;
};

__global__ void k_sub_rows(SubRowsArgs S)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < S.m; j += warps) {
        const int64_t i = S.idx[j];
        const int64_t p0 = S.indptr[i], len = S.indptr[i + 1] - p0, q0 = S.sub_indptr[j];
        for (int64_t k = lane; k < len; k += 32) {
            S.sub_indices[q0 + k] = S.indices[p0 + k];
            if (S.sub_values) S.sub_values[q0 + k] = S.values[p0 + k];
            if (S.sub_vmix) S.sub_vmix[q0 + k] = S.vmix[p0 + k];
            if (S.sub_ew) S.sub_ew[q0 + k] = S.ew[p0 + k];
            if (S.sub_ew64) S.sub_ew64[q0 + k] = S.ew64[p0 + k];
        }
        for (int k = lane; k < S.bit_words; k += 32) S.sub_bits[j * S.bit_words + k] = S.bits[i * S.bit_words + k];
        if (S.dmat) {
            const uint4 *src = reinterpret_cast<const uint4 *>(S.dmat + i * S.d_pad);
            uint4 *dst = reinterpret_cast<uint4 *>(S.sub_dmat + j * S.d_pad);
            for (int k = lane; k < S.d_pad / 8; k += 32) dst[k] = src[k];
        }
        if (lane == 0) {
            S.sub_y[j] = S.y[i];
            if (S.sub_norm) S.sub_norm[j] = S.norm[i];
            if (S.sub_normf) S.sub_normf[j] = S.normf[i];
            S.sub_alpha[j] = S.alpha[i];
            S.sub_f[j] = S.f[i];
            S.sub_status[j] = S.status[i];
            S.sub_gmap[j] = S.pmap ? S.pmap[i] : (int32_t)i;
        }
    }
}

// solver state of the smaller problem back into its parent; mark[i] = 1 for
// the parent rows still active
__global__ void k_sub_scatter(int64_t m, const int32_t *idx, const double *sub_alpha, const double *sub_f,
                              const uint8_t *sub_status, const uint8_t *sub_mark, double *alpha, double *f,
                              uint8_t *status, uint8_t *mark)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    const int64_t i = idx[j];
    alpha[i] = sub_alpha[j];
    f[i] = sub_f[j];
    status[i] = sub_status[j];
    mark[i] = sub_mark[j];
}

// active lists from marks: segment s lists its marked rows in increasing
// order (one block of 256 threads per segment)
__global__ void k_active_from_mark(int64_t n, int G, const uint8_t *mark, int32_t *act, int32_t *seg_cnt)
{
    __shared__ int wsum[8];
    __shared__ int base;
    const int s = blockIdx.x, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t lo = seg_lo(n, G, s);
    const int m = (int)(seg_lo(n, G, s + 1) - lo);
    if (threadIdx.x == 0) base = 0;
    __syncthreads();
    for (int r0 = 0; r0 < m; r0 += 256) {
        const int r = r0 + threadIdx.x;
        const bool p = r < m && mark[lo + r] != 0;
        const unsigned bal = __ballot_sync(0xffffffffu, p);
        if (lane == 0) wsum[w] = __popc(bal);
        __syncthreads();
        int pre = base + __popc(bal & ((1u << lane) - 1u));
        int tot = 0;
        for (int k = 0; k < 8; ++k) {
            if (k < w) pre += wsum[k];
            tot += wsum[k];
        }
        if (p) act[lo + pre] = r;
        __syncthreads();
        if (threadIdx.x == 0) base += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) seg_cnt[s] = base;
}

// ---- deterministic, order-preserving compaction by predicate
enum { PRED_UNMARKED = 0, PRED_ALPHA_POS = 1, PRED_MARKED = 2 };
constexpr int kChunk = 4096;
constexpr int kCT = 256;

__device__ __forceinline__ bool pred_at(int pred, int64_t i, const uint8_t *mark, const double *alpha)
{
    return pred == PRED_UNMARKED ? mark[i] == 0 : (pred == PRED_MARKED ? mark[i] != 0 : alpha[i] > 0.0);
}

__global__ void k_count(int pred, int64_t n, const uint8_t *mark, const double *alpha, int *counts)
{
    __shared__ int s;
    if (threadIdx.x == 0) s = 0;
    __syncthreads();
    int64_t b0 = (int64_t)blockIdx.x * kChunk;
    int c = 0;
    for (int64_t i = b0 + threadIdx.x; i < n && i < b0 + kChunk; i += kCT) c += pred_at(pred, i, mark, alpha);
    atomicAdd(&s, c);
    __syncthreads();
    if (threadIdx.x == 0) counts[blockIdx.x] = s;
}

__global__ void k_scan(const int *counts, int nb, int *offsets, long long *total)
{
    if (threadIdx.x != 0) return;
    long long acc = 0;
    for (int b = 0; b < nb; ++b) {
        offsets[b] = (int)acc;
        acc += counts[b];
    }
    *total = acc;
}

__global__ void k_scatter(int pred, int64_t n, const uint8_t *mark, const double *alpha,
                          const int8_t *y, const int *offsets, int32_t *list, double *coef)
{
    __shared__ int wsum[kCT / 32];
    __shared__ int base;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x == 0) base = offsets[blockIdx.x];
    __syncthreads();
    int64_t b0 = (int64_t)blockIdx.x * kChunk;
    for (int64_t s0 = b0; s0 < n && s0 < b0 + kChunk; s0 += kCT) {
        int64_t i = s0 + threadIdx.x;
        bool p = i < n && i < b0 + kChunk && pred_at(pred, i, mark, alpha);
        unsigned m = __ballot_sync(0xffffffffu, p);
        if (lane == 0) wsum[w] = __popc(m);
        __syncthreads();
        int pre = __popc(m & ((1u << lane) - 1u));
        for (int k = 0; k < w; ++k) pre += wsum[k];
        int tot = 0;
        for (int k = 0; k < kCT / 32; ++k) tot += wsum[k];
        if (p) {
            list[base + pre] = (int32_t)i;
            if (coef) coef[base + pre] = alpha[i] * (double)y[i];
        }
        __syncthreads();
        if (threadIdx.x == 0) base += tot;
        __syncthreads();
    }
}

// ---- final reductions (fixed order): objective, threshold b, counts
struct FinishPart {
    double sum_a;        // sum alpha
    double sum_ayfy;     // sum alpha_i y_i (f_i + y_i)
    double sum_f0;       // sum f over I0
    long long n0, nsv, nbound;
};

__global__ void k_finish_part(int64_t n, double C, const double *alpha, const double *f,
                              const uint8_t *status, FinishPart *parts)
{
    __shared__ FinishPart sp[kCT];
    int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
    int64_t b0 = (int64_t)blockIdx.x * chunk, b1 = min(n, b0 + chunk);
    FinishPart p = {0, 0, 0, 0, 0, 0};
    for (int64_t i = b0 + threadIdx.x; i < b1; i += kCT) {
        double a = alpha[i];
        uint8_t sb = status[i];
        double yi = (sb & 0x80) ? 1.0 : -1.0;
        p.sum_a += a;
        p.sum_ayfy += a * yi * (f[i] + yi);
        if ((sb & 7) == ST_I0) {
            p.sum_f0 += f[i];
            p.n0 += 1;
        }
        if (a > 0.0) p.nsv += 1;
        if (a == C) p.nbound += 1;
    }
    sp[threadIdx.x] = p;
    __syncthreads();
    for (int s = kCT / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
            FinishPart &a = sp[threadIdx.x];
            const FinishPart &b = sp[threadIdx.x + s];
            a.sum_a += b.sum_a;
            a.sum_ayfy += b.sum_ayfy;
            a.sum_f0 += b.sum_f0;
            a.n0 += b.n0;
            a.nsv += b.nsv;
            a.nbound += b.nbound;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) parts[blockIdx.x] = sp[0];
}

__global__ void k_finish_total(const FinishPart *parts, int nb, FinishPart *out)
{
    if (threadIdx.x != 0) return;
    FinishPart t = {0, 0, 0, 0, 0, 0};
    for (int b = 0; b < nb; ++b) {
        t.sum_a += parts[b].sum_a;
        t.sum_ayfy += parts[b].sum_ayfy;
        t.sum_f0 += parts[b].sum_f0;
        t.n0 += parts[b].n0;
        t.nsv += parts[b].nsv;
        t.nbound += parts[b].nbound;
    }
    *out = t;
}

// --------------------------------------------------------------- helpers

int grid1(int64_t n, int t = 256) { return (int)((n + t - 1) / t); }

int device_sms()
{
    int dev = 0, sms = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    return sms;
}

// Device-resident copy of one CSR matrix (+ labels) with its derived data.
// Binary rows as bit masks of W words: bit c of row i is set when column c
// is stored (d <= 32 W).
__global__ void k_bits(int64_t n, int W, const int64_t *indptr, const int32_t *indices, uint32_t *bits)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t m[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int64_t p = indptr[i]; p < indptr[i + 1]; ++p) {
        const int c = indices[p];
        m[(c >> 5) & 7] |= 1u << (c & 31);
    }
    for (int w = 0; w < W; ++w) bits[i * W + w] = m[w];
}

struct DevCSR {
    int64_t n = 0, d = 0, nnz = 0;
    const int64_t *indptr = nullptr;
    const int32_t *indices = nullptr;
    const float *values = nullptr;   // NULL for binary input
    const int8_t *y = nullptr;
    double *norm = nullptr;
    float *vmix = nullptr;
    float *normf = nullptr;
    bool binary = false;
    int maxnnz = 0;
    int64_t npos = 0;
    const IngestInfo *info = nullptr;   // the validation record (device)
    XdFormat xd{};                      // exact inner products of the matrix with itself
    int bmax = 0, bmin = 255;           // exponent range of the nonzero values
    bool subnormal = false;
};

// The exact-inner-product format for products between two matrices.
XdFormat xd_pair(const DevCSR &A, const DevCSR &B)
{
    return xd_format(std::max(A.bmax, B.bmax), std::min(A.bmin, B.bmin), std::max(A.maxnnz, B.maxnnz),
                     A.subnormal || B.subnormal);
}

__global__ void k_fill_ones(int64_t m, float *v)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) v[i] = 1.0f;
}

// binary_ok = false: binary rows are kept on the general (values) path,
// with explicit 1.0 values when the matrix has none
void ingest(Arena &ar, const svm_csr *X, const int8_t *y, bool need_fp64, bool need_mixed,
            cudaStream_t st, DevCSR &out, int *launches, bool binary_ok = true)
{
    if (!X) ARG_FAIL("matrix is NULL");
    if (X->n < 1 || X->d < 1) ARG_FAIL("n and d must be >= 1 (n=%lld d=%lld)", (long long)X->n, (long long)X->d);
    if (X->n >= (int64_t)INT32_MAX) ARG_FAIL("n must be < 2^31");
    if (X->d >= (int64_t)INT32_MAX) ARG_FAIL("d must be < 2^31");
    if (!X->indptr || (!X->indices && X->n > 0)) ARG_FAIL("indptr/indices must not be NULL");
    out.n = X->n;
    out.d = X->d;
    int64_t nnz = 0;
    if (X->on_device) {
        CK(cudaMemcpyAsync(&nnz, X->indptr + X->n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
    } else {
        nnz = X->indptr[X->n];
    }
    if (nnz < 0 || nnz >= ((int64_t)1 << 40)) ARG_FAIL("indptr[n] out of range");
    out.nnz = nnz;
    if (X->on_device) {
        out.indptr = X->indptr;
        out.indices = X->indices;
        out.values = X->values;
        out.y = y;
    } else {
        int64_t *ip = ar.alloc<int64_t>(X->n + 1);
        CK(cudaMemcpyAsync(ip, X->indptr, sizeof(int64_t) * (X->n + 1), cudaMemcpyHostToDevice, st));
        int32_t *ix = ar.alloc<int32_t>(nnz);
        if (nnz) CK(cudaMemcpyAsync(ix, X->indices, sizeof(int32_t) * nnz, cudaMemcpyHostToDevice, st));
        out.indptr = ip;
        out.indices = ix;
        if (X->values) {
            float *v = ar.alloc<float>(nnz);
            if (nnz) CK(cudaMemcpyAsync(v, X->values, sizeof(float) * nnz, cudaMemcpyHostToDevice, st));
            out.values = v;
        }
        if (y) {
            int8_t *yd = ar.alloc<int8_t>(X->n);
            CK(cudaMemcpyAsync(yd, y, X->n, cudaMemcpyHostToDevice, st));
            out.y = yd;
        }
    }
    IngestInfo *info = ar.alloc<IngestInfo>(1);
    CK(cudaMemsetAsync(info, 0, sizeof(IngestInfo), st));
    k_validate<<<grid1(X->n), 256, 0, st>>>(X->n, X->d, out.indptr, out.indices, out.values, out.y, info);
    CK(cudaGetLastError());
    ++*launches;
    IngestInfo h;
    CK(cudaMemcpyAsync(&h, info, sizeof h, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (h.bad_indptr) ARG_FAIL("indptr is not non-decreasing from 0");
    if (h.bad_index) ARG_FAIL("column indices must be strictly increasing within a row and < d");
    if (h.nonfinite) ARG_FAIL("values must be finite");
    if (y && h.bad_y) ARG_FAIL("labels must be +1 or -1");
    out.binary = !h.not_binary;
    if (out.binary && !binary_ok) {
        out.binary = false;
        if (!out.values && nnz > 0) {
            float *v = ar.alloc<float>(nnz);
            k_fill_ones<<<grid1(nnz), 256, 0, st>>>(nnz, v);
            CK(cudaGetLastError());
            ++*launches;
            out.values = v;
        }
    }
    out.maxnnz = h.maxnnz;
    out.npos = (int64_t)h.npos;
    out.info = info;
    // input without values: every value is 1.0 (b = 127), filled or not
    out.bmax = X->values ? h.bmax : 127;
    out.bmin = X->values ? 255 - h.nbmin : 127;
    out.subnormal = X->values && h.subnormal != 0;
    out.xd = xd_format(out.bmax, out.bmin, out.maxnnz, out.subnormal);
    if (!out.binary && need_fp64) out.norm = ar.alloc<double>(X->n);
    if (!out.binary && need_mixed) {
        out.vmix = ar.alloc<float>(nnz);
        out.normf = ar.alloc<float>(X->n);
    }
    if (out.norm || out.vmix) {
        k_norms<<<grid1(X->n), 256, 0, st>>>(X->n, out.indptr, out.values, out.norm, out.vmix, out.normf, info);
        CK(cudaGetLastError());
        ++*launches;
    }
}

cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

// order-preserving compaction; returns the count
int64_t compact(Arena &ar, int pred, int64_t n, const uint8_t *mark, const double *alpha,
                const int8_t *y, int32_t *list, double *coef, cudaStream_t st, int *launches)
{
    int nb = (int)((n + kChunk - 1) / kChunk);
    int *counts = ar.alloc<int>(nb);
    int *offs = ar.alloc<int>(nb);
    long long *tot = ar.alloc<long long>(1);
    k_count<<<nb, kCT, 0, st>>>(pred, n, mark, alpha, counts);
    k_scan<<<1, 32, 0, st>>>(counts, nb, offs, tot);
    k_scatter<<<nb, kCT, 0, st>>>(pred, n, mark, alpha, y, offs, list, coef);
    CK(cudaGetLastError());
    *launches += 3;
    long long h = 0;
    CK(cudaMemcpyAsync(&h, tot, sizeof h, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return h;
}

size_t smem_limit()
{
    int dev = 0, v = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    return (size_t)v;
}

double elapsed_ms(std::chrono::steady_clock::time_point t0)
{
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

int train_impl(const svm_csr *X, const int8_t *y, const svm_params *P, const svm_shrink_policy *pol,
               double *alpha_out, double *b_out, int64_t *iters_out, svm_stats *stats)
{
    auto t_start = std::chrono::steady_clock::now();
    if (!P) ARG_FAIL("params is NULL");
    if (!y) ARG_FAIL("labels are NULL");
    if (!alpha_out || !b_out) ARG_FAIL("alpha_out and b_out must not be NULL");
    if (!(P->C > 0) || !std::isfinite(P->C)) ARG_FAIL("C must be > 0");
    if (!(P->gamma > 0) || !std::isfinite(P->gamma)) ARG_FAIL("gamma must be > 0");
    if (!(P->tau > 0) || !std::isfinite(P->tau)) ARG_FAIL("tau must be > 0");
    if (P->precision < SVM_FP64 || P->precision > SVM_MIXED_BF16_SIMT) ARG_FAIL("unknown precision %d", P->precision);
    if (P->tie_break != 0) ARG_FAIL("only the lowest-index tie-break (0) is implemented");
    if (X && X->n < 2) ARG_FAIL("need at least two samples");
    svm_shrink_policy none = {SVM_SHRINK_NONE, SVM_RECON_SINGLE, 0.0, 20.0};
    const svm_shrink_policy &sp = pol ? *pol : none;
    if (sp.kind < SVM_SHRINK_NONE || sp.kind > SVM_SHRINK_FRACTION) ARG_FAIL("unknown shrink kind %d", sp.kind);
    if (sp.recon != SVM_RECON_SINGLE && sp.recon != SVM_RECON_MULTI) ARG_FAIL("unknown reconstruction mode %d", sp.recon);
    if (sp.kind != SVM_SHRINK_NONE && !(sp.value > 0)) ARG_FAIL("shrink value must be > 0");
    if (P->kernel < SVM_KERNEL_RBF || P->kernel > SVM_KERNEL_SIGMOID) ARG_FAIL("unknown kernel %d", P->kernel);
    if (P->kernel == SVM_KERNEL_POLY && (P->degree < 1 || P->degree > 64)) ARG_FAIL("polynomial degree must be 1..64");
    if (!std::isfinite(P->coef0)) ARG_FAIL("coef0 must be finite");
    const bool rbf = P->kernel == SVM_KERNEL_RBF;
    cudaStream_t st = as_stream(P->stream);
    int launches = 0;
    Arena ar(st);
    DevCSR D;
    const bool mixed = P->precision != SVM_FP64;
    const bool use_tc = P->precision == SVM_MIXED_BF16 && rbf;
    ingest(ar, X, y, !mixed, mixed, st, D, &launches, rbf);
    const int64_t n = D.n;
    if (D.npos == 0 || D.npos == n) ARG_FAIL("both classes must be present");

    // row-pass arithmetic and its shared-memory footprint
    int mode = D.binary ? MODE_BINARY : (mixed ? MODE_MIXED : MODE_FP64);
    int ktab_len = 2 * D.maxnnz + 1;
    const size_t lim = smem_limit() - 8192;
    if (mode == MODE_BINARY && smo_layout(MODE_BINARY, (int)D.d, ktab_len, D.maxnnz, 0, 0, 0).total > lim) {
        // too many columns for the binary tables: use the generic path,
        // with explicit 1.0 values when the matrix has none
        mode = mixed ? MODE_MIXED : MODE_FP64;
        if (!D.values && D.nnz > 0) {
            float *v = ar.alloc<float>(D.nnz);
            k_fill_ones<<<grid1(D.nnz), 256, 0, st>>>(D.nnz, v);
            CK(cudaGetLastError());
            ++launches;
            D.values = v;
        }
        if (mode == MODE_FP64 && !D.norm) D.norm = ar.alloc<double>(n);
        if (mode == MODE_MIXED && !D.vmix) {
            D.vmix = ar.alloc<float>(D.nnz);
            D.normf = ar.alloc<float>(n);
        }
        k_norms<<<grid1(n), 256, 0, st>>>(n, D.indptr, D.values, D.norm, D.vmix, D.normf, D.info);
        CK(cudaGetLastError());
        ++launches;
    }
    // lanes per row from the mean row length; one CTA per SM
    double avg = (double)D.nnz / (double)n;
    // one thread per row up to 32 stored entries (the f updates then run on
    // full warps of the weak FP64 pipe), more lanes for longer rows
    int lpr = 1;
    while (lpr < 32 && lpr * 32 < avg) lpr <<= 1;
    if (P->lanes_per_row > 0) {
        lpr = 1;
        while (lpr < 32 && lpr < P->lanes_per_row) lpr <<= 1;
    }
    // binary rows with d <= 256: bit masks, one lane per row
    int kmode = mode;
    uint32_t *bits = nullptr;
    if (mode == MODE_BINARY && D.d <= 256 && (P->flags & SVM_FLAG_CSR_ROWS) == 0) {
        kmode = D.d <= 128 ? MODE_BITS4 : MODE_BITS8;
        lpr = 1;
        const int W = mode_words(kmode);
        bits = ar.alloc<uint32_t>((size_t)n * W);
        k_bits<<<grid1(n), 256, 0, st>>>(n, W, D.indptr, D.indices, bits);
        CK(cudaGetLastError());
        ++launches;
    }
    // mixed mode, RBF, d <= 256: kernel rows on the tensor cores (16-row
    // tiles against the two targets) from a dense BF16 copy of the rows.
    // Automatic for rows that are dense enough and not too wide (measured:
    // d = 64 and 128 dense 2.3x and 1.4x faster per step than the CSR pass
    // on the CUDA cores; d = 20 and 256 dense and the covtype-shaped 12 of
    // 54 columns slower), or forced on / off by the flags.
    const int d_pad = (int)((D.d + 31) / 32 * 32);
    const double avg_nnz = (double)D.nnz / (double)n;
    const bool tiles_ok = kmode == MODE_MIXED && use_tc && D.d <= 256 && P->cache_mb <= 0 &&
                          (P->flags & SVM_FLAG_CUDA_CORE_ROWS) == 0;
    const bool row_tiles = tiles_ok && ((P->flags & SVM_FLAG_TENSOR_ROWS) != 0 ||
                                        (d_pad <= 128 && avg_nnz >= 32.0 && avg_nnz >= 0.5 * d_pad));
    __nv_bfloat16 *dmat = nullptr;
    if (row_tiles) {
        lpr = 16;
        dmat = ar.alloc<__nv_bfloat16>((size_t)n * d_pad);
        k_dense_bf16<<<(unsigned)n, 128, 0, st>>>(n, (int)D.d, d_pad, D.indptr, D.indices, D.vmix, dmat);
        CK(cudaGetLastError());
        ++launches;
    }
    const int sms = device_sms();
    const int kt = mode == MODE_BINARY ? ktab_len : 0;
    const size_t lim_dyn = smem_limit() - smo_static_smem(kmode) - 1024;
    // kernel-row cache (FP64 and mixed inputs): every slot holds one kernel
    // row over all n samples; all n rows when they fit (direct), else up to
    // 8192 rows in 4-way sets; the directory goes into each CTA's shared
    // memory, so its size is part of the layout
    // The plan is made again for every level of the active-set re-layout
    // (below) within the buffer sized at the top level: rows of a smaller
    // level are shorter, so more of them fit, and the whole kernel matrix of
    // the small late levels fits directly.
    struct KcPlan {
        int64_t ld = 0;
        int slots = 0, direct = 0;
    };
    const size_t kc_esz = kmode == MODE_FP64 ? 8 : 4;
    auto plan_kc = [&](int64_t n_l, size_t cap) {
        KcPlan k;
        k.ld = (n_l + 31) / 32 * 32;
        const size_t row_bytes = (size_t)k.ld * kc_esz;
        if ((size_t)n_l * row_bytes <= cap && smo_kdir_bytes(n_l, 0, 1) <= lim_dyn / 4) {
            k.slots = (int)n_l;
            k.direct = 1;
        } else {
            int64_t sl = std::min<int64_t>((int64_t)(cap / row_bytes), 8192);
            while (sl >= 64 && smo_kdir_bytes(n_l, (int)sl, 0) > lim_dyn / 2) sl /= 2;
            k.slots = sl >= 64 ? (int)(sl / 4 * 4) : 0;
        }
        return k;
    };
    KcPlan top_kc;
    size_t kc_cap = 0;   // bytes of the cache buffer
    size_t kdir = 0;
    // automatic for FP64 rows (their exp costs ~20 FP64 instructions per
    // value); the mixed mode's FP32 exp is cheaper than the cache traffic, so
    // there the cache is used only when a budget is given
    if ((kmode == MODE_FP64 && P->cache_mb >= 0) || (kmode == MODE_MIXED && P->cache_mb > 0)) {
        size_t budget = (size_t)P->cache_mb << 20;
        if (P->cache_mb == 0) {
            size_t fr = 0, tot = 0;
            if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) fr = 0;
            budget = std::min<size_t>(fr / 2, (size_t)32 << 30);
        }
        top_kc = plan_kc(n, budget);
        if (top_kc.slots > 0) {
            kc_cap = (size_t)top_kc.slots * (size_t)top_kc.ld * kc_esz;
            kdir = smo_kdir_bytes(n, top_kc.slots, top_kc.direct);
        }
    }
    const int kc_slots = top_kc.slots, kc_direct = top_kc.direct;
    const int64_t kc_ld = top_kc.ld;
    // launch shape of a problem of n_l rows and nnz_l entries (the caller's
    // problem, or the active rows gathered after shrinking): thread-block
    // clusters for the hierarchical exchange, one cluster of 16 when its
    // segments stay in shared memory (no global exchange at all), else
    // clusters of 8 with a leader exchange through global memory; segment
    // sizes decide whether the rows stay in shared memory
    struct Shape {
        int G, cs, resident, seg_rows_max;
        int64_t seg_nnz_max;
        size_t smem;
    };
    int64_t *segnnz_d = ar.alloc<int64_t>(256);
    auto pick_shape = [&](int64_t n_l, int64_t nnz_l, const int64_t *indptr_l, size_t kdir_l) -> Shape {
        int G_l = (int)std::min<int64_t>(sms, std::max<int64_t>(1, (n_l + 15) / 16));
        if (P->ctas > 0) G_l = (int)std::min<int64_t>(std::min<int64_t>(P->ctas, sms), n_l);
        if (G_l > 256) G_l = 256;
        int cs_l = 1;
        const SmoLayout L0 = smo_layout(kmode, (int)D.d, kt, D.maxnnz, 0, 0, 0, kdir_l);
        const bool clusters_ok = (P->flags & SVM_FLAG_NO_CLUSTERS) == 0 && L0.total <= lim_dyn;
        bool single = false;
        if (clusters_ok && (P->ctas == 0 || P->ctas == 16) && n_l >= 16 * 32 &&
            (P->flags & SVM_FLAG_STREAM_ROWS) == 0) {
            const int rows16 = (int)((n_l + 15) / 16);
            const int64_t nnz16 = (int64_t)(1.25 * (double)nnz_l / 16.0) + D.maxnnz;   // segment estimate
            const SmoLayout L16 = smo_layout(kmode, (int)D.d, kt, D.maxnnz, 1, rows16, nnz16, kdir_l);
            // FP64 rows cost ~50 operations of the FP64 pipe each (about two
            // issue per clock per SM here), so above a few thousand rows 16 SMs
            // are slower than clusters of 8 over the whole GPU despite their
            // cheaper exchange (measured crossover ~7,000 covtype-shaped rows)
            const int64_t one_cluster_max = kmode == MODE_FP64 ? kFp64OneClusterRows : 200000;
            if (L16.total <= lim_dyn && smo_max_clusters(kmode, lpr, 2, L16.total, 16) >= 1 &&
                (P->ctas == 16 || n_l <= one_cluster_max)) {
                single = true;
                cs_l = 16;
                G_l = 16;
            }
        }
        if (!single && clusters_ok && G_l >= 16) {
            const int maxc = smo_max_clusters(kmode, lpr, 0, L0.total, 8);
            if (maxc >= 2) {
                cs_l = 8;
                G_l = 8 * std::min(maxc, G_l / 8);
            }
        }
        int64_t seg_nnz_max_l = 0;
        int seg_rows_max_l = 0;
        SmoLayout Ls{}, Lr{};
        int resident_l = 0;
        for (int pass = 0; pass < 2; ++pass) {
            k_seg_nnz<<<grid1(G_l), 256, 0, st>>>(n_l, G_l, indptr_l, segnnz_d);
            CK(cudaGetLastError());
            ++launches;
            std::vector<int64_t> segnnz(G_l);
            CK(cudaMemcpyAsync(segnnz.data(), segnnz_d, sizeof(int64_t) * G_l, cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            seg_nnz_max_l = 0;
            for (int64_t v : segnnz) seg_nnz_max_l = std::max(seg_nnz_max_l, v);
            seg_rows_max_l = (int)((n_l + G_l - 1) / G_l);
            Ls = smo_layout(kmode, (int)D.d, kt, D.maxnnz, 0, seg_rows_max_l, seg_nnz_max_l, kdir_l);
            Lr = smo_layout(kmode, (int)D.d, kt, D.maxnnz, 1, seg_rows_max_l, seg_nnz_max_l, kdir_l);
            resident_l = (P->flags & SVM_FLAG_STREAM_ROWS) == 0 && D.d <= 65535 &&
                         seg_nnz_max_l < ((int64_t)1 << 31) && Lr.total <= lim_dyn;
            if (resident_l && cs_l > 1 &&
                smo_max_clusters(kmode, lpr, G_l == cs_l ? 2 : 1, Lr.total, cs_l) * cs_l < G_l)
                resident_l = 0;
            if (resident_l || cs_l != 16) break;
            // the single cluster was chosen for on-chip segments that do not
            // fit after all: clusters of 8 over the whole GPU instead
            cs_l = 8;
            const size_t s0 = smo_layout(kmode, (int)D.d, kt, D.maxnnz, 0, 0, 0, kdir_l).total;
            G_l = 8 * std::max(1, std::min(smo_max_clusters(kmode, lpr, 0, s0, 8), std::min(sms, 256) / 8));
        }
        // Rows that stream from global memory, and FP64 levels of many rows,
        // are bound by the row pass, not by the exchange: there one CTA on
        // every SM with the flat exchange beats clusters of 8, which leave the
        // SMs that do not make up whole clusters idle (measured on GB300:
        // covtype-shaped full set 87 -> 71 us/step FP64, 28 -> 25 mixed)
        if (P->ctas == 0 && cs_l == 8 && (!resident_l || (kmode == MODE_FP64 && n_l >= kFp64FlatRows))) {
            const int Gf = (int)std::min<int64_t>(std::min(sms, 256), std::max<int64_t>(1, (n_l + 15) / 16));
            k_seg_nnz<<<grid1(Gf), 256, 0, st>>>(n_l, Gf, indptr_l, segnnz_d);
            CK(cudaGetLastError());
            ++launches;
            std::vector<int64_t> segnnz(Gf);
            CK(cudaMemcpyAsync(segnnz.data(), segnnz_d, sizeof(int64_t) * Gf, cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            int64_t snm = 0;
            for (int64_t v : segnnz) snm = std::max(snm, v);
            const int srm = (int)((n_l + Gf - 1) / Gf);
            const SmoLayout Lsf = smo_layout(kmode, (int)D.d, kt, D.maxnnz, 0, srm, snm, kdir_l);
            const SmoLayout Lrf = smo_layout(kmode, (int)D.d, kt, D.maxnnz, 1, srm, snm, kdir_l);
            const int resf = (P->flags & SVM_FLAG_STREAM_ROWS) == 0 && D.d <= 65535 &&
                             snm < ((int64_t)1 << 31) && Lrf.total <= lim_dyn;
            if ((resf ? Lrf.total : Lsf.total) <= lim_dyn) {
                G_l = Gf;
                cs_l = 1;
                resident_l = resf;
                seg_rows_max_l = srm;
                seg_nnz_max_l = snm;
                Ls = Lsf;
                Lr = Lrf;
            }
        }
        Shape sh;
        sh.G = G_l;
        sh.cs = cs_l;
        sh.resident = resident_l;
        sh.seg_rows_max = seg_rows_max_l;
        sh.seg_nnz_max = seg_nnz_max_l;
        sh.smem = resident_l ? Lr.total : Ls.total;
        if (sh.smem > lim_dyn) {
            set_err("d = %lld exceeds the shared-memory target rows of this mode", (long long)D.d);
            throw Fail{SVM_ERR_UNSUPPORTED};
        }
        return sh;
    };
    const Shape top = pick_shape(n, D.nnz, D.indptr, kdir);
    const int G = top.G;
    const int cs = top.cs, resident = top.resident;
    double *ktab = nullptr;
    if (mode == MODE_BINARY) {
        ktab = ar.alloc<double>(3 * (size_t)ktab_len);
        k_ktab<<<grid1(ktab_len), 256, 0, st>>>(P->gamma, ktab_len, ktab);
        CK(cudaGetLastError());
        ++launches;
    }
    const float *vals_fp32 = D.values;

    // solver state
    double *alpha = ar.alloc<double>(n);
    double *f = ar.alloc<double>(n);
    uint8_t *status = ar.alloc<uint8_t>(n);
    int32_t *act = ar.alloc<int32_t>(n);
    int32_t *seg_cnt = ar.alloc<int32_t>(256);
    // exchange slots and flags for the largest grid of any level (<= 256 CTAs)
    void *cand = ar.alloc<unsigned char>(smo_cand_slots(256) * smo_cand_bytes());
    unsigned *seq = ar.alloc<unsigned>(smo_seq_words(256));
    SmoCtrl *ctrl = ar.alloc<SmoCtrl>(1);
    const int64_t trace_len = (P->trace && P->trace_len > 0) ? P->trace_len : 0;
    int32_t *trace = ar.alloc<int32_t>(2 * std::max<int64_t>(trace_len, 1));
    if (trace_len) CK(cudaMemsetAsync(trace, 0xff, sizeof(int32_t) * 2 * trace_len, st));
    const int64_t atrace_len = (P->active_trace && P->active_trace_len > 0) ? P->active_trace_len : 0;
    int64_t *atrace = ar.alloc<int64_t>(2 * std::max<int64_t>(atrace_len, 1));
    if (atrace_len) CK(cudaMemsetAsync(atrace, 0xff, sizeof(int64_t) * 2 * atrace_len, st));
    k_init<<<grid1(n), 256, 0, st>>>(n, D.y, alpha, f, status);
    k_reset_active<<<G, 256, 0, st>>>(n, G, act, seg_cnt);
    CK(cudaGetLastError());
    launches += 2;

    // warm start (resume): alpha0 checked on the host, index sets from it, and
    // f = sum_j alpha_j y_j K(x_i, x_j) - y_i (Eq. fcache) by the contraction
    // that reconstruction uses (support vectors = alpha0 > 0, queries = all)
    if (P->alpha0) {
        std::vector<double> a0(n);
        std::vector<int8_t> yh(n);
        CK(cudaMemcpyAsync(a0.data(), P->alpha0, sizeof(double) * n,
                           X->on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost, st));
        CK(cudaMemcpyAsync(yh.data(), D.y, n, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        double ysum = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            if (!(a0[i] >= 0.0 && a0[i] <= P->C)) ARG_FAIL("alpha0[%lld] is outside [0, C]", (long long)i);
            ysum += yh[i] > 0 ? a0[i] : -a0[i];
        }
        if (!(std::fabs(ysum) <= 1e-9 * std::max(1.0, P->C * (double)n)))
            ARG_FAIL("alpha0 violates sum y alpha = 0 (%.3g)", ysum);
        double *a0d = ar.alloc<double>(n);
        CK(cudaMemcpyAsync(a0d, a0.data(), sizeof(double) * n, cudaMemcpyHostToDevice, st));
        k_init_warm<<<grid1(n), 256, 0, st>>>(n, P->C, D.y, a0d, alpha, status);
        CK(cudaGetLastError());
        ++launches;
        int32_t *w_sv = ar.alloc<int32_t>(n);
        double *w_coef = ar.alloc<double>(n);
        const int64_t w_nsv = compact(ar, PRED_ALPHA_POS, n, nullptr, alpha, D.y, w_sv, w_coef, st, &launches);
        if (w_nsv > 0) {
            int32_t *w_q = ar.alloc<int32_t>(n);
            k_iota<<<grid1(n), 256, 0, st>>>(n, w_q);
            CK(cudaGetLastError());
            ++launches;
            RbfContract c;
            std::memset(&c, 0, sizeof c);
            c.x_indptr = D.indptr;
            c.x_indices = D.indices;
            c.x_values = mode == MODE_MIXED ? D.vmix : D.values;
            c.x_norm = D.norm;
            c.x_normf = D.normf;
            c.sv = w_sv;
            c.coef = w_coef;
            c.nsv = w_nsv;
            c.z_indptr = D.indptr;
            c.z_indices = D.indices;
            c.z_values = c.x_values;
            c.z_norm = D.norm;
            c.z_normf = D.normf;
            c.q = w_q;
            c.nq = n;
            c.d = (int32_t)D.d;
            c.mode = mode;
            c.gamma = P->gamma;
            c.kernel = P->kernel;
            c.degree = P->degree;
            c.coef0 = P->coef0;
            c.ktab = ktab;
            c.ktab_len = ktab_len;
            c.out_by_row = 1;
            c.out = f;
            c.yq = D.y;
            c.add_scalar = 0.0;
            c.xd = D.xd;
            if (use_tc && mode == MODE_MIXED && tc_rbf_supported((int)D.d)) {
                void *ws = ar.alloc<unsigned char>(tc_rbf_workspace_bytes(n, w_nsv, (int)D.d));
                int tc_err = 0;
                CK(launch_rbf_contract_tc(c, ws, &tc_err, st));
                launches += 3;
                CK(cudaStreamSynchronize(st));
                if (tc_err) {
                    set_err("a wait in the tensor-core contraction exceeded its limit");
                    throw Fail{SVM_ERR_TIMEOUT};
                }
            } else {
                CK(launch_rbf_contract(c, st));
                ++launches;
            }
        }
    }

    const bool shrink_on = sp.kind != SVM_SHRINK_NONE;
    int64_t h = 0;
    if (sp.kind == SVM_SHRINK_FIXED) h = (int64_t)sp.value;
    if (sp.kind == SVM_SHRINK_FRACTION) h = (int64_t)std::ceil(sp.value * (double)n);
    if (shrink_on && h < 1) h = 1;
    const double ff = sp.first_factor > 0 ? sp.first_factor : 20.0;
    const int64_t max_iter = P->max_iter > 0 ? P->max_iter : 100 * n + 1000000;

    SmoCtrl hc;
    std::memset(&hc, 0, sizeof hc);
    hc.counter = h;
    hc.active = n;
    hc.i_up = hc.i_low = -1;

    SmoArgs A;
    std::memset(&A, 0, sizeof A);
    A.n = n;
    A.d = (int32_t)D.d;
    A.G = G;
    A.indptr = D.indptr;
    A.indices = D.indices;
    A.values = vals_fp32;
    A.vmix = D.vmix;
    A.y = D.y;
    A.norm = D.norm;
    A.normf = D.normf;
    A.bits = bits;
    A.alpha = alpha;
    A.f = f;
    A.status = status;
    A.act = act;
    A.seg_cnt = seg_cnt;
    A.cand = cand;
    A.seq = seq;
    A.ctrl = ctrl;
    A.trace = trace;
    A.trace_len = trace_len;
    A.atrace = atrace;
    A.atrace_len = atrace_len;
    A.ktab = ktab;
    A.ktab_len = ktab_len;
    A.maxnnz = D.maxnnz;
    A.xd = D.xd;
    A.resident = resident;
    A.seg_rows_max = top.seg_rows_max;
    A.seg_nnz_max = top.seg_nnz_max;
    A.C = P->C;
    A.gamma = P->gamma;
    A.phase_times = (P->flags & SVM_FLAG_PHASE_TIMES) != 0;
    A.wss2 = (P->flags & SVM_FLAG_WSS2) != 0;
    A.kernel = P->kernel;
    A.degree = P->degree;
    A.coef0 = P->coef0;
    void *kc_buf = kc_cap ? ar.alloc<unsigned char>(kc_cap) : nullptr;
    if (kc_slots > 0) {
        A.kc = kc_buf;
        A.kc_ld = kc_ld;
        A.kc_slots = kc_slots;
        A.kc_direct = kc_direct;
    }
    int64_t *cta_cycles = nullptr;
    if (A.phase_times) {
        cta_cycles = ar.alloc<int64_t>(256);
        CK(cudaMemsetAsync(cta_cycles, 0, sizeof(int64_t) * 256, st));
    }
    A.cta_cycles = cta_cycles;
    A.timeout_ns = 10ll * 1000 * 1000 * 1000;

    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    double ms_smo = 0.0, ms_recon = 0.0;
    // Active-set re-layout (with shrinking): a launch over a problem that is
    // not already one on-chip cluster ends once a quarter of its rows have
    // been shrunk (measured: 3.47 -> 3.29 s against waiting for half of them
    // on the covtype-shaped workload, no gain from waiting for an eighth); the active rows are gathered, in index order, into a
    // smaller problem whose launch shape is chosen again (segments on chip,
    // a single cluster), and its state is scattered back when its launch
    // ends. Rows keep their order, so every step is the one the parent
    // problem would have taken (the same pairs, the same arithmetic).
    struct Level {
        int64_t n, nnz;
        const int64_t *indptr;
        const int32_t *indices;
        const float *values, *vmix, *normf;
        const double *norm;
        const int8_t *y;
        const uint32_t *bits;
        double *alpha, *f;
        uint8_t *status;
        int32_t *act, *seg_cnt;
        const int32_t *idx;    // this level's rows in its parent (NULL at the top)
        const int32_t *gmap;   // ... and in the caller's problem
        Shape shape;
        const __nv_bfloat16 *dmat;   // dense BF16 rows for the row tiles, or NULL
        KcPlan kc;                   // kernel-row cache plan of this level
        const uint32_t *ew;          // mixed rows one word per entry (d < 2^16), or NULL
        const uint64_t *ew64;        // FP64 rows with exact inner products, packed entries, or NULL
    };
    const bool relayout_on = (P->flags & SVM_FLAG_NO_RELAYOUT) == 0;
    bool relayout_ok = relayout_on;
    const int bit_words = mode_bits(kmode) ? mode_words(kmode) : 0;
    // mixed rows: one word per stored entry (column and BF16 value), which
    // the row pass loads once instead of the column and the value; required
    // for rows held on chip, which need d < 2^16 anyway
    uint32_t *ew = nullptr;
    if (kmode == MODE_MIXED && D.d <= 65535 && D.vmix && D.nnz > 0) {
        ew = ar.alloc<uint32_t>(D.nnz);
        k_pack_ew<<<grid1(D.nnz), 256, 0, st>>>(D.nnz, D.indices, D.vmix, ew);
        CK(cudaGetLastError());
        ++launches;
    }
    // FP64 rows with exact inner products: column and (m, b - t) word in one
    // 8-byte entry, which the streamed row pass loads once
    uint64_t *ew64 = nullptr;
    if (kmode == MODE_FP64 && D.xd.on && D.d <= 65535 && vals_fp32 && D.nnz > 0) {
        ew64 = ar.alloc<uint64_t>(D.nnz);
        k_pack_ew64<<<grid1(D.nnz), 256, 0, st>>>(D.nnz, D.indices, vals_fp32, D.xd.tmin, ew64);
        CK(cudaGetLastError());
        ++launches;
    }
    std::vector<Level> lv;
    lv.push_back(Level{n, D.nnz, D.indptr, D.indices, vals_fp32, D.vmix, D.normf, D.norm, D.y, bits,
                       alpha, f, status, act, seg_cnt, nullptr, nullptr, top, dmat, top_kc, ew, ew64});
    int64_t relayouts = 0;
    auto launch_level = [&](const Level &L, int select_only, double thr, int64_t hh, int64_t limit) {
        A.n = L.n;
        A.G = L.shape.G;
        A.indptr = L.indptr;
        A.indices = L.indices;
        A.values = L.values;
        A.vmix = L.vmix;
        A.ew = L.ew;
        A.ew64 = L.ew64;
        A.y = L.y;
        A.norm = L.norm;
        A.normf = L.normf;
        A.bits = L.bits;
        A.alpha = L.alpha;
        A.f = L.f;
        A.status = L.status;
        A.act = L.act;
        A.seg_cnt = L.seg_cnt;
        A.resident = L.shape.resident;
        A.seg_rows_max = L.shape.seg_rows_max;
        A.seg_nnz_max = L.shape.seg_nnz_max;
        A.gmap = L.gmap;
        A.dmat = L.dmat;
        A.d_pad = d_pad;
        A.kc = L.kc.slots > 0 ? kc_buf : nullptr;
        A.kc_ld = L.kc.ld;
        A.kc_slots = L.kc.slots;
        A.kc_direct = L.kc.direct;
        const bool one_cluster_on_chip = L.shape.resident && L.shape.cs == L.shape.G;
        A.compact_below = (relayout_ok && hh > 0 && !one_cluster_on_chip && L.n >= 2048) ? L.n * 3 / 4 : 0;
        CK(cudaMemcpyAsync(ctrl, &hc, sizeof hc, cudaMemcpyHostToDevice, st));
        CK(cudaMemsetAsync(seq, 0, sizeof(unsigned) * smo_seq_words(L.shape.G), st));
        // tagged slots: a word of an earlier launch must not carry this one's epochs
        CK(cudaMemsetAsync(cand, 0, smo_cand_slots(L.shape.G) * smo_cand_bytes(), st));
        A.thr = thr;
        A.h = hh;
        A.iter_limit = limit;
        A.select_only = select_only;
        CK(cudaEventRecord(e0, st));
        CK(launch_smo_persistent(kmode, lpr, A, L.shape.smem, st, L.shape.cs));
        CK(cudaEventRecord(e1, st));
        ++launches;
        CK(cudaMemcpyAsync(&hc, ctrl, sizeof hc, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        ms_smo += ms;
        if (hc.err) {
            set_err("a grid-wide wait in the SMO kernel exceeded its time limit");
            throw Fail{SVM_ERR_TIMEOUT};
        }
    };
    // the active rows of the deepest level into a new level; false when
    // there are too few of them to be worth it
    auto push_level = [&]() -> bool {
        const Level Pa = lv.back();
        uint8_t *mk = ar.alloc<uint8_t>(Pa.n);
        CK(cudaMemsetAsync(mk, 0, Pa.n, st));
        k_mark_active<<<Pa.shape.G, 256, 0, st>>>(Pa.n, Pa.shape.G, Pa.act, Pa.seg_cnt, mk);
        CK(cudaGetLastError());
        ++launches;
        int32_t *idx = ar.alloc<int32_t>(Pa.n);
        const int64_t m = compact(ar, PRED_MARKED, Pa.n, mk, nullptr, nullptr, idx, nullptr, st, &launches);
        if (m < 2 * 32) return false;
        const int nb = (int)((m + kChunkRows - 1) / kChunkRows);
        int64_t *sums = ar.alloc<int64_t>(nb);
        int64_t *offs = ar.alloc<int64_t>(nb);
        int64_t *tot = ar.alloc<int64_t>(1);
        int64_t *sub_indptr = ar.alloc<int64_t>(m + 1);
        k_sub_len_sums<<<nb, 256, 0, st>>>(m, idx, Pa.indptr, sums);
        k_scan64<<<1, 32, 0, st>>>(sums, nb, offs, tot);
        k_sub_indptr<<<nb, 256, 0, st>>>(m, idx, Pa.indptr, offs, sub_indptr);
        CK(cudaGetLastError());
        launches += 3;
        int64_t nnz_m = 0;
        CK(cudaMemcpyAsync(&nnz_m, tot, sizeof nnz_m, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        SubRowsArgs S;
        std::memset(&S, 0, sizeof S);
        S.m = m;
        S.idx = idx;
        S.pmap = Pa.gmap;
        S.indptr = Pa.indptr;
        S.indices = Pa.indices;
        S.values = Pa.values;
        S.vmix = Pa.vmix;
        S.normf = Pa.normf;
        S.norm = Pa.norm;
        S.alpha = Pa.alpha;
        S.f = Pa.f;
        S.y = Pa.y;
        S.status = Pa.status;
        S.bits = Pa.bits;
        S.bit_words = Pa.bits ? bit_words : 0;
        S.sub_indptr = sub_indptr;
        S.sub_indices = ar.alloc<int32_t>(nnz_m);
        // only the values the row pass reads: FP32 (FP64 mode) or BF16-rounded (mixed)
        S.sub_values = (Pa.values && kmode == MODE_FP64) ? ar.alloc<float>(nnz_m) : nullptr;
        S.sub_vmix = (Pa.vmix && kmode == MODE_MIXED) ? ar.alloc<float>(nnz_m) : nullptr;
        S.ew = Pa.ew;
        S.sub_ew = Pa.ew ? ar.alloc<uint32_t>(nnz_m) : nullptr;
        S.ew64 = Pa.ew64;
        S.sub_ew64 = Pa.ew64 ? ar.alloc<uint64_t>(nnz_m) : nullptr;
        S.sub_normf = Pa.normf ? ar.alloc<float>(m) : nullptr;
        S.sub_norm = Pa.norm ? ar.alloc<double>(m) : nullptr;
        S.sub_alpha = ar.alloc<double>(m);
        S.sub_f = ar.alloc<double>(m);
        S.sub_y = ar.alloc<int8_t>(m);
        S.sub_status = ar.alloc<uint8_t>(m);
        S.sub_bits = S.bit_words ? ar.alloc<uint32_t>((size_t)m * S.bit_words) : nullptr;
        S.sub_gmap = ar.alloc<int32_t>(m);
        S.dmat = Pa.dmat;
        S.sub_dmat = Pa.dmat ? ar.alloc<__nv_bfloat16>((size_t)m * d_pad) : nullptr;
        S.d_pad = d_pad;
        k_sub_rows<<<(int)std::min<int64_t>((m + 7) / 8, 4096), 256, 0, st>>>(S);
        CK(cudaGetLastError());
        ++launches;
        Level C;
        C.n = m;
        C.nnz = nnz_m;
        C.indptr = sub_indptr;
        C.indices = S.sub_indices;
        C.values = S.sub_values;
        C.vmix = S.sub_vmix;
        C.normf = S.sub_normf;
        C.norm = S.sub_norm;
        C.y = S.sub_y;
        C.bits = S.sub_bits;
        C.alpha = S.sub_alpha;
        C.f = S.sub_f;
        C.status = S.sub_status;
        C.act = ar.alloc<int32_t>(m);
        C.seg_cnt = ar.alloc<int32_t>(256);
        C.idx = idx;
        C.gmap = S.sub_gmap;
        C.dmat = S.sub_dmat;
        C.ew = S.sub_ew;
        C.ew64 = S.sub_ew64;
        C.kc = kc_cap ? plan_kc(m, kc_cap) : KcPlan{};
        C.shape = pick_shape(m, nnz_m, sub_indptr, C.kc.slots > 0 ? smo_kdir_bytes(m, C.kc.slots, C.kc.direct) : 0);
        k_reset_active<<<C.shape.G, 256, 0, st>>>(m, C.shape.G, C.act, C.seg_cnt);
        CK(cudaGetLastError());
        ++launches;
        lv.push_back(C);
        ++relayouts;
        return true;
    };
    // the deepest level's state back into its parent
    auto pop_level = [&]() {
        const Level C = lv.back();
        lv.pop_back();
        const Level &Pa = lv.back();
        uint8_t *cm = ar.alloc<uint8_t>(C.n);
        uint8_t *pm = ar.alloc<uint8_t>(Pa.n);
        CK(cudaMemsetAsync(cm, 0, C.n, st));
        CK(cudaMemsetAsync(pm, 0, Pa.n, st));
        k_mark_active<<<C.shape.G, 256, 0, st>>>(C.n, C.shape.G, C.act, C.seg_cnt, cm);
        k_sub_scatter<<<grid1(C.n), 256, 0, st>>>(C.n, C.idx, C.alpha, C.f, C.status, cm, Pa.alpha, Pa.f,
                                                  Pa.status, pm);
        k_active_from_mark<<<Pa.shape.G, 256, 0, st>>>(Pa.n, Pa.shape.G, pm, Pa.act, Pa.seg_cnt);
        CK(cudaGetLastError());
        launches += 3;
    };
    // Incremental reconstruction: when a run's launch over the caller's
    // problem ends at its first shrink event and its active rows are gathered
    // into a level, the rows shrunk there hold f exact at that moment, and
    // afterwards only the gathered rows' alpha change. Their f at the end is
    // then that f plus the contraction over the gathered rows whose alpha
    // changed (Algorithm 6's sum over all support vectors, less the terms
    // whose alpha did not change since f was exact). inc_*: the gather.
    bool inc_track = false, inc_ok = false;
    const int32_t *inc_idx = nullptr;
    int64_t inc_m = 0;
    double *inc_a0 = nullptr;
    auto run = [&](int select_only, double thr, int64_t hh, int64_t limit) {
        int sel = select_only;
        bool top = true;
        if (inc_track) inc_ok = false;
        for (;;) {
            const int64_t se0 = hc.shrink_events;
            launch_level(lv.back(), sel, thr, hh, limit);
            if (hc.exit_reason != 2) break;
            const bool one_event = top && hc.shrink_events - se0 == 1;
            // the same state continues on the gathered rows (a selection
            // pass there finds the pair this launch had chosen)
            if (!push_level()) {
                relayout_ok = false;
            } else if (inc_track && one_event && lv.size() == 2) {
                const Level &Cl = lv.back();
                inc_idx = Cl.idx;
                inc_m = Cl.n;
                inc_a0 = ar.alloc<double>(inc_m);
                CK(cudaMemcpyAsync(inc_a0, Cl.alpha, sizeof(double) * inc_m, cudaMemcpyDeviceToDevice, st));
                inc_ok = true;
            }
            top = false;
            sel = 1;
        }
        while (lv.size() > 1) pop_level();
        relayout_ok = relayout_on;
    };

    bool shrinking = shrink_on;
    double thr = shrinking ? ff * P->tau : 2.0 * P->tau;
    int64_t n_recon = 0;
    int status_code = SVM_OK;
    uint8_t *mark = nullptr;
    int32_t *list_w = nullptr, *list_sv = nullptr;
    double *coef = nullptr;
    // the CUDA-core contraction can add to f (the tensor-core one writes it)
    const bool inc_allowed = (P->flags & SVM_FLAG_FULL_RECON) == 0 && !(use_tc && mode == MODE_MIXED);
    int64_t inc_recons = 0;
    for (;;) {
        inc_track = inc_allowed && shrinking;
        run(1, thr, shrinking ? h : 0, max_iter);
        inc_track = false;
        if (hc.exit_reason == 1) {
            status_code = SVM_NOT_CONVERGED;
            break;
        }
        if (!shrinking) break;
        // Algorithm 6: reconstruct f of the shrunk samples from all alpha > 0
        if (hc.active < n) {
            if (!mark) {
                mark = ar.alloc<uint8_t>(n);
                list_w = ar.alloc<int32_t>(n);
                list_sv = ar.alloc<int32_t>(n);
                coef = ar.alloc<double>(n);
            }
            CK(cudaEventRecord(e0, st));
            CK(cudaMemsetAsync(mark, 0, n, st));
            k_mark_active<<<G, 256, 0, st>>>(n, G, act, seg_cnt, mark);
            CK(cudaGetLastError());
            ++launches;
            // incremental part: rows shrunk at the gather get f += the
            // contraction over the gathered rows whose alpha changed
            int64_t inc_nq = 0, inc_nd = 0;
            int32_t *inc_q = nullptr, *inc_list = nullptr;
            double *inc_coef = nullptr;
            const uint8_t *full_mark = mark;
            if (inc_ok) {
                uint8_t *gathered = ar.alloc<uint8_t>(n), *dmark = ar.alloc<uint8_t>(n);
                uint8_t *q1 = ar.alloc<uint8_t>(n), *q2 = ar.alloc<uint8_t>(n);
                double *dalpha = ar.alloc<double>(n);
                CK(cudaMemsetAsync(gathered, 0, n, st));
                CK(cudaMemsetAsync(dmark, 0, n, st));
                CK(cudaMemsetAsync(dalpha, 0, sizeof(double) * n, st));
                k_inc_delta<<<grid1(inc_m), 256, 0, st>>>(inc_m, inc_idx, inc_a0, alpha, dalpha, dmark, gathered);
                k_inc_marks<<<grid1(n), 256, 0, st>>>(n, mark, gathered, q1, q2);
                CK(cudaGetLastError());
                launches += 2;
                inc_q = ar.alloc<int32_t>(n);
                inc_list = ar.alloc<int32_t>(n);
                inc_coef = ar.alloc<double>(n);
                inc_nq = compact(ar, PRED_UNMARKED, n, q1, alpha, D.y, inc_q, nullptr, st, &launches);
                inc_nd = compact(ar, PRED_MARKED, n, dmark, dalpha, D.y, inc_list, inc_coef, st, &launches);
                full_mark = q2;   // the full sum only for the gathered rows shrunk later
                ++inc_recons;
            }
            int64_t nw = compact(ar, PRED_UNMARKED, n, full_mark, alpha, D.y, list_w, nullptr, st, &launches);
            int64_t nsv = nw > 0 ? compact(ar, PRED_ALPHA_POS, n, mark, alpha, D.y, list_sv, coef, st, &launches) : 0;
            RbfContract c;
            std::memset(&c, 0, sizeof c);
            c.x_indptr = D.indptr;
            c.x_indices = D.indices;
            c.x_values = mode == MODE_MIXED ? D.vmix : D.values;
            c.x_norm = D.norm;
            c.x_normf = D.normf;
            c.sv = list_sv;
            c.coef = coef;
            c.nsv = nsv;
            c.z_indptr = D.indptr;
            c.z_indices = D.indices;
            c.z_values = c.x_values;
            c.z_norm = D.norm;
            c.z_normf = D.normf;
            c.q = list_w;
            c.nq = nw;
            c.d = (int32_t)D.d;
            c.mode = mode;
            c.gamma = P->gamma;
            c.kernel = P->kernel;
            c.degree = P->degree;
            c.coef0 = P->coef0;
            c.ktab = ktab;
            c.ktab_len = ktab_len;
            c.out_by_row = 1;
            c.out = f;
            c.yq = D.y;
            c.add_scalar = 0.0;
            c.xd = D.xd;
            if (use_tc && mode == MODE_MIXED && nsv > 0 && tc_rbf_supported((int)D.d)) {
                void *ws = ar.alloc<unsigned char>(tc_rbf_workspace_bytes(nw, nsv, (int)D.d));
                int tc_err = 0;
                CK(launch_rbf_contract_tc(c, ws, &tc_err, st));
                launches += 3;
                CK(cudaStreamSynchronize(st));
                if (tc_err) {
                    set_err("a wait in the tensor-core reconstruction exceeded its limit");
                    throw Fail{SVM_ERR_TIMEOUT};
                }
            } else if (nw > 0) {
                CK(launch_rbf_contract(c, st));
                ++launches;
            }
            if (inc_nq > 0 && inc_nd > 0) {
                c.sv = inc_list;
                c.coef = inc_coef;
                c.nsv = inc_nd;
                c.q = inc_q;
                c.nq = inc_nq;
                c.yq = nullptr;
                c.accumulate = 1;
                CK(launch_rbf_contract(c, st));
                ++launches;
            }
            CK(cudaEventRecord(e1, st));
            CK(cudaStreamSynchronize(st));
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, e0, e1));
            ms_recon += ms;
        }
        ++n_recon;
        k_reset_active<<<G, 256, 0, st>>>(n, G, act, seg_cnt);
        CK(cudaGetLastError());
        ++launches;
        hc.active = n;
        // b_up / b_low over all samples (a selection pass, no steps)
        run(1, 2.0 * P->tau, 0, hc.iter);
        if (!(hc.b_low - hc.b_up > 2.0 * P->tau)) break;
        if (sp.recon == SVM_RECON_SINGLE) shrinking = false;
        else hc.counter = h;
        thr = 2.0 * P->tau;
    }

    // threshold b (Section III-A), objective, counts
    const int nbf = (int)std::min<int64_t>(1024, std::max<int64_t>(1, (n + 4095) / 4096));
    FinishPart *parts = ar.alloc<FinishPart>(nbf);
    FinishPart *tot = ar.alloc<FinishPart>(1);
    k_finish_part<<<nbf, kCT, 0, st>>>(n, P->C, alpha, f, status, parts);
    k_finish_total<<<1, 32, 0, st>>>(parts, nbf, tot);
    CK(cudaGetLastError());
    launches += 2;
    FinishPart fp;
    CK(cudaMemcpyAsync(&fp, tot, sizeof fp, cudaMemcpyDeviceToHost, st));
    if (X->on_device) CK(cudaMemcpyAsync(alpha_out, alpha, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    else CK(cudaMemcpyAsync(alpha_out, alpha, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
    std::vector<int32_t> tr;
    if (trace_len) {
        tr.resize(2 * trace_len);
        CK(cudaMemcpyAsync(tr.data(), trace, sizeof(int32_t) * 2 * trace_len, cudaMemcpyDeviceToHost, st));
    }
    if (atrace_len)
        CK(cudaMemcpyAsync(P->active_trace, atrace, sizeof(int64_t) * 2 * atrace_len, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (trace_len) {
        for (int64_t t = 0; t < trace_len; ++t) {
            bool done = t < hc.iter;
            P->trace[2 * t] = done ? tr[2 * t] : -1;
            P->trace[2 * t + 1] = done ? tr[2 * t + 1] : -1;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const double b = fp.n0 > 0 ? fp.sum_f0 / (double)fp.n0 : 0.5 * (hc.b_up + hc.b_low);
    *b_out = b;
    if (iters_out) *iters_out = hc.iter;
    if (stats) {
        stats->iters = hc.iter;
        stats->shrink_events = hc.shrink_events;
        stats->reconstructions = n_recon;
        stats->incremental_recons = (int32_t)inc_recons;
        stats->final_active = hc.active;
        stats->n_sv = fp.nsv;
        stats->n_bound = fp.nbound;
        stats->row_visits = hc.row_visits;
        stats->b_up = hc.b_up;
        stats->b_low = hc.b_low;
        stats->objective = fp.sum_a - 0.5 * fp.sum_ayfy;
        stats->ms_smo = ms_smo;
        stats->ms_recon = ms_recon;
        stats->binary_input = mode == MODE_BINARY;
        stats->resident = resident;
        stats->ctas = G;
        stats->cluster_size = cs;
        stats->lanes_per_row = lpr;
        stats->bit_rows = mode_bits(kmode) ? 1 : 0;
        stats->cache_slots = kc_slots;
        stats->cache_hits = hc.kc_hits;
        stats->cache_misses = hc.kc_misses;
        stats->relayouts = relayouts;
        stats->row_tiles = row_tiles ? 1 : 0;
        int dev = 0, khz = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev);
        for (int k = 0; k < 8; ++k) stats->phase_ms[k] = khz > 0 ? (double)hc.phase_cycles[k] / (double)khz : 0.0;
        stats->cta_busy_ms_min = stats->cta_busy_ms_max = 0.0;
        if (cta_cycles && khz > 0) {
            std::vector<int64_t> cc(G);
            CK(cudaMemcpy(cc.data(), cta_cycles, sizeof(int64_t) * G, cudaMemcpyDeviceToHost));
            int64_t mn = cc[0], mx = cc[0];
            for (int64_t v : cc) { mn = std::min(mn, v); mx = std::max(mx, v); }
            stats->cta_busy_ms_min = (double)mn / khz;
            stats->cta_busy_ms_max = (double)mx / khz;
        }
        stats->launches = launches;
        stats->ms_total = elapsed_ms(t_start);
    }
    g_launches += launches;
    return status_code;
}

void check_kernel(const svm_kernel &K)
{
    if (!(K.gamma > 0)) ARG_FAIL("gamma must be > 0");
    if (K.kind < SVM_KERNEL_RBF || K.kind > SVM_KERNEL_SIGMOID) ARG_FAIL("unknown kernel %d", K.kind);
    if (K.kind == SVM_KERNEL_POLY && (K.degree < 1 || K.degree > 64)) ARG_FAIL("polynomial degree must be 1..64");
    if (!std::isfinite(K.coef0)) ARG_FAIL("coef0 must be finite");
}

// Eq. (classi) before the sign for the queries Z against support vectors:
// rows list_sv[0 .. nsv) of DX with coefficients coef (alpha y). DX was
// ingested for this precision; it is taken by value because norms it lacks
// are derived into the call's arena.
void decision_eval(Arena &ar, DevCSR DX, const int32_t *list_sv, const double *coef, int64_t nsv, double b,
                   const svm_kernel &K, const svm_csr *Z, int32_t precision, cudaStream_t st, double *out,
                   int *launches_out)
{
    int launches = 0;
    const bool rbf = K.kind == SVM_KERNEL_RBF;
    const bool mixed = precision != SVM_FP64;
    DevCSR DZ;
    ingest(ar, Z, nullptr, !mixed, mixed, st, DZ, &launches, rbf);
    int mode = (DX.binary && DZ.binary) ? MODE_BINARY : (mixed ? MODE_MIXED : MODE_FP64);
    if (mode != MODE_BINARY && (DX.binary || DZ.binary)) {
        // one side binary, the other not: derive the missing norms
        for (DevCSR *D : {&DX, &DZ}) {
            if (mode == MODE_FP64 && !D->norm) D->norm = ar.alloc<double>(D->n);
            if (mode == MODE_MIXED && !D->vmix) {
                D->vmix = ar.alloc<float>(D->nnz);
                D->normf = ar.alloc<float>(D->n);
            }
            k_norms<<<grid1(D->n), 256, 0, st>>>(D->n, D->indptr, D->values, D->norm, D->vmix, D->normf, D->info);
            CK(cudaGetLastError());
            ++launches;
        }
    }
    int ktab_len = DX.maxnnz + DZ.maxnnz + 1;
    double *ktab = nullptr;
    if (mode == MODE_BINARY) {
        ktab = ar.alloc<double>(3 * (size_t)ktab_len);
        k_ktab<<<grid1(ktab_len), 256, 0, st>>>(K.gamma, ktab_len, ktab);
        CK(cudaGetLastError());
        ++launches;
    }
    size_t need = mode == MODE_BINARY ? 4 * (size_t)DX.d : (mode == MODE_FP64 ? 8 * 8 : 4 * 8) * (size_t)DX.d;
    if (need > smem_limit() - 8192) {
        set_err("d = %lld exceeds the shared-memory query tile of this mode", (long long)DX.d);
        throw Fail{SVM_ERR_UNSUPPORTED};
    }
    double *out_d = out;
    if (!Z->on_device) out_d = ar.alloc<double>(DZ.n);
    RbfContract c;
    std::memset(&c, 0, sizeof c);
    c.x_indptr = DX.indptr;
    c.x_indices = DX.indices;
    c.x_values = mode == MODE_MIXED ? DX.vmix : DX.values;
    c.x_norm = DX.norm;
    c.x_normf = DX.normf;
    c.sv = list_sv;
    c.coef = coef;
    c.nsv = nsv;
    c.z_indptr = DZ.indptr;
    c.z_indices = DZ.indices;
    c.z_values = mode == MODE_MIXED ? DZ.vmix : DZ.values;
    c.z_norm = DZ.norm;
    c.z_normf = DZ.normf;
    c.q = nullptr;
    c.nq = DZ.n;
    c.d = (int32_t)DX.d;
    c.mode = mode;
    c.gamma = K.gamma;
    c.kernel = K.kind;
    c.degree = K.degree;
    c.coef0 = K.coef0;
    c.ktab = ktab;
    c.ktab_len = ktab_len;
    c.out_by_row = 0;
    c.out = out_d;
    c.yq = nullptr;
    c.add_scalar = -b;
    c.xd = xd_pair(DX, DZ);
    if (rbf && precision == SVM_MIXED_BF16 && mode == MODE_MIXED && nsv > 0 && tc_rbf_supported((int)DX.d)) {
        void *ws = ar.alloc<unsigned char>(tc_rbf_workspace_bytes(DZ.n, nsv, (int)DX.d));
        int tc_err = 0;
        CK(launch_rbf_contract_tc(c, ws, &tc_err, st));
        launches += 3;
        CK(cudaStreamSynchronize(st));
        if (tc_err) {
            set_err("a wait in the tensor-core decision kernel exceeded its limit");
            throw Fail{SVM_ERR_TIMEOUT};
        }
    } else {
        CK(launch_rbf_contract(c, st));
        ++launches;
    }
    if (!Z->on_device) CK(cudaMemcpyAsync(out, out_d, sizeof(double) * DZ.n, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    *launches_out += launches;
}

int decision_impl(const svm_csr *X, const int8_t *y, const double *alpha, double b, const svm_kernel &K,
                  const svm_csr *Z, int32_t precision, void *stream, double *out)
{
    if (!X || !Z || !y || !alpha || !out) ARG_FAIL("NULL argument");
    check_kernel(K);
    const bool rbf = K.kind == SVM_KERNEL_RBF;
    if (Z->d != X->d) ARG_FAIL("Z->d (%lld) must equal X->d (%lld)", (long long)Z->d, (long long)X->d);
    if (precision < SVM_FP64 || precision > SVM_MIXED_BF16_SIMT) ARG_FAIL("unknown precision %d", precision);
    if (Z->n == 0) return SVM_OK;
    cudaStream_t st = as_stream(stream);
    int launches = 0;
    Arena ar(st);
    const bool mixed = precision != SVM_FP64;
    DevCSR DX;
    ingest(ar, X, y, !mixed, mixed, st, DX, &launches, rbf);
    const int64_t n = DX.n;
    const double *alpha_d = alpha;
    if (!X->on_device) {
        double *a = ar.alloc<double>(n);
        CK(cudaMemcpyAsync(a, alpha, sizeof(double) * n, cudaMemcpyHostToDevice, st));
        alpha_d = a;
    }
    int32_t *list_sv = ar.alloc<int32_t>(n);
    double *coef = ar.alloc<double>(n);
    int64_t nsv = compact(ar, PRED_ALPHA_POS, n, nullptr, alpha_d, DX.y, list_sv, coef, st, &launches);
    decision_eval(ar, DX, list_sv, coef, nsv, b, K, Z, precision, st, out, &launches);
    g_launches += launches;
    return SVM_OK;
}

// ---------------------------------------------------------------------------
// Trained model held on the device: the support vectors (rows with alpha > 0,
// gathered in index order into their own CSR), alpha y and b, so that
// decisions on new queries re-read neither the training rows nor alpha.
// ---------------------------------------------------------------------------

// rows idx[0 .. m) of a CSR (entries, values, norms) into a compact CSR
struct GatherArgs {
    int64_t m;
    const int32_t *idx;
    const int64_t *indptr;
    const int32_t *indices;
    const float *values, *vmix, *normf;
    const double *norm;
    const int64_t *sub_indptr;
    int32_t *sub_indices;
    float *sub_values, *sub_vmix, *sub_normf;
    double *sub_norm;
};

__global__ void k_gather_rows(GatherArgs S)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < S.m; j += warps) {
        const int64_t i = S.idx[j];
        const int64_t p0 = S.indptr[i], len = S.indptr[i + 1] - p0, q0 = S.sub_indptr[j];
        for (int64_t k = lane; k < len; k += 32) {
            S.sub_indices[q0 + k] = S.indices[p0 + k];
            if (S.sub_values) S.sub_values[q0 + k] = S.values[p0 + k];
            if (S.sub_vmix) S.sub_vmix[q0 + k] = S.vmix[p0 + k];
        }
        if (lane == 0) {
            if (S.sub_norm) S.sub_norm[j] = S.norm[i];
            if (S.sub_normf) S.sub_normf[j] = S.normf[i];
        }
    }
}

struct ModelState {
    int device = 0;
    DevCSR sv;                      // support-vector rows (model-owned memory)
    int32_t *list = nullptr;        // 0 .. nsv-1
    double *coef = nullptr;         // alpha y of each support vector
    int64_t nsv = 0;
    double b = 0.0;
    svm_kernel K{};
    int32_t precision = SVM_FP64;
    std::vector<void *> mem;        // device allocations freed with the model
};

ModelState *model_create_impl(const svm_csr *X, const int8_t *y, const double *alpha, double b,
                              const svm_kernel &K, int32_t precision, void *stream)
{
    if (!X || !y || !alpha) ARG_FAIL("NULL argument");
    check_kernel(K);
    if (precision < SVM_FP64 || precision > SVM_MIXED_BF16_SIMT) ARG_FAIL("unknown precision %d", precision);
    if (!std::isfinite(b)) ARG_FAIL("b must be finite");
    cudaStream_t st = as_stream(stream);
    int launches = 0;
    const bool rbf = K.kind == SVM_KERNEL_RBF;
    const bool mixed = precision != SVM_FP64;
    Arena ar(st);     // scratch of this call
    Arena keep(st);   // what the model keeps (handed over below)
    DevCSR DX;
    ingest(ar, X, y, !mixed, mixed, st, DX, &launches, rbf);
    const int64_t n = DX.n;
    const double *alpha_d = alpha;
    if (!X->on_device) {
        double *a = ar.alloc<double>(n);
        CK(cudaMemcpyAsync(a, alpha, sizeof(double) * n, cudaMemcpyHostToDevice, st));
        alpha_d = a;
    }
    int32_t *list = ar.alloc<int32_t>(n);
    double *coef_all = ar.alloc<double>(n);
    const int64_t m = compact(ar, PRED_ALPHA_POS, n, nullptr, alpha_d, DX.y, list, coef_all, st, &launches);
    std::unique_ptr<ModelState> M(new ModelState());
    CK(cudaGetDevice(&M->device));
    M->nsv = m;
    M->b = b;
    M->K = K;
    M->precision = precision;
    DevCSR S;
    S.n = m;
    S.d = DX.d;
    S.binary = DX.binary;
    S.maxnnz = DX.maxnnz;
    int64_t *sub_indptr = keep.alloc<int64_t>(m + 1);
    int64_t nnz_m = 0;
    if (m > 0) {
        const int nb = (int)((m + kChunkRows - 1) / kChunkRows);
        int64_t *sums = ar.alloc<int64_t>(nb);
        int64_t *offs = ar.alloc<int64_t>(nb);
        int64_t *tot = ar.alloc<int64_t>(1);
        k_sub_len_sums<<<nb, 256, 0, st>>>(m, list, DX.indptr, sums);
        k_scan64<<<1, 32, 0, st>>>(sums, nb, offs, tot);
        k_sub_indptr<<<nb, 256, 0, st>>>(m, list, DX.indptr, offs, sub_indptr);
        CK(cudaGetLastError());
        launches += 3;
        CK(cudaMemcpyAsync(&nnz_m, tot, sizeof nnz_m, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
    } else {
        CK(cudaMemsetAsync(sub_indptr, 0, sizeof(int64_t), st));
    }
    S.nnz = nnz_m;
    GatherArgs G;
    std::memset(&G, 0, sizeof G);
    G.m = m;
    G.idx = list;
    G.indptr = DX.indptr;
    G.indices = DX.indices;
    G.values = DX.values;
    G.vmix = DX.vmix;
    G.normf = DX.normf;
    G.norm = DX.norm;
    G.sub_indptr = sub_indptr;
    G.sub_indices = keep.alloc<int32_t>(nnz_m);
    G.sub_values = DX.values ? keep.alloc<float>(nnz_m) : nullptr;
    G.sub_vmix = DX.vmix ? keep.alloc<float>(nnz_m) : nullptr;
    G.sub_normf = DX.normf ? keep.alloc<float>(m) : nullptr;
    G.sub_norm = DX.norm ? keep.alloc<double>(m) : nullptr;
    if (m > 0) {
        k_gather_rows<<<(int)std::min<int64_t>((m + 7) / 8, 4096), 256, 0, st>>>(G);
        CK(cudaGetLastError());
        ++launches;
    }
    S.indptr = sub_indptr;
    S.indices = G.sub_indices;
    S.values = G.sub_values;
    S.vmix = G.sub_vmix;
    S.normf = G.sub_normf;
    S.norm = G.sub_norm;
    M->sv = S;
    M->coef = keep.alloc<double>(std::max<int64_t>(m, 1));
    M->list = keep.alloc<int32_t>(std::max<int64_t>(m, 1));
    if (m > 0) {
        CK(cudaMemcpyAsync(M->coef, coef_all, sizeof(double) * m, cudaMemcpyDeviceToDevice, st));
        k_iota<<<grid1(m), 256, 0, st>>>(m, M->list);
        CK(cudaGetLastError());
        ++launches;
    }
    CK(cudaStreamSynchronize(st));
    M->mem = std::move(keep.ptrs);
    keep.ptrs.clear();
    g_launches += launches;
    return M.release();
}

void model_free_impl(ModelState *M)
{
    if (!M) return;
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != M->device) cudaSetDevice(M->device);
    for (void *p : M->mem) cudaFree(p);
    if (cur != M->device) cudaSetDevice(cur);
    delete M;
}

// ---------------------------------------------------------------------------
// Batched training (many subproblems over one matrix in one launch)
// ---------------------------------------------------------------------------

// BF16 dense copy of dense rows (row stride d_pad, zero padding).
__global__ void k_dense_bf16(int64_t n, int d, int d_pad, const int64_t *indptr, const int32_t *indices,
                             const float *vmix, __nv_bfloat16 *out)
{
    const int64_t r = blockIdx.x;
    if (r >= n) return;
    __nv_bfloat16 *dst = out + (size_t)r * d_pad;
    for (int c = threadIdx.x; c < d_pad; c += blockDim.x) dst[c] = __float2bfloat16_rn(0.f);
    __syncthreads();
    for (int64_t p = indptr[r] + threadIdx.x; p < indptr[r + 1]; p += blockDim.x)
        dst[indices[p]] = __float2bfloat16_rn(vmix[p]);
}

__global__ void k_iota(int64_t n, int32_t *out)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (int32_t)i;
}

// per job: row ids in range, labels +-1, both classes present
__global__ void k_job_check(int njobs, const BatchJobDev *jobs, int64_t n, int *bad)
{
    const int j = blockIdx.x;
    if (j >= njobs) return;
    __shared__ int s_bad, s_pos, s_neg;
    if (threadIdx.x == 0) s_bad = s_pos = s_neg = 0;
    __syncthreads();
    const BatchJobDev J = jobs[j];
    int b = 0, pos = 0, neg = 0;
    for (int r = threadIdx.x; r < J.nrows; r += blockDim.x) {
        const int32_t g = J.rows[r];
        const int8_t v = J.y[r];
        if (g < 0 || g >= n) b = 1;
        if (v == 1) pos = 1;
        else if (v == -1) neg = 1;
        else b = 1;
    }
    if (b) atomicOr(&s_bad, 1);
    if (pos) atomicOr(&s_pos, 1);
    if (neg) atomicOr(&s_neg, 1);
    __syncthreads();
    if (threadIdx.x == 0) bad[j] = s_bad ? 1 : ((s_pos && s_neg) ? 0 : 2);
}

struct BatchPlan {
    DevCSR D;
    int mode = MODE_FP64;
    int dense = 0;
    int d_eff = 0;
    __nv_bfloat16 *dense_rows = nullptr;
    int ktab_len = 0;
    size_t smem = 0;
};

void batch_prepare(Arena &ar, const svm_csr *X, int precision, cudaStream_t st, BatchPlan &B, int *launches)
{
    const bool mixed = precision != SVM_FP64;
    ingest(ar, X, nullptr, !mixed, mixed, st, B.D, launches);
    DevCSR &D = B.D;
    B.mode = D.binary ? MODE_BINARY : (mixed ? MODE_MIXED : MODE_FP64);
    if (B.mode == MODE_BINARY && smo_layout(MODE_BINARY, (int)D.d, 2 * D.maxnnz + 1, D.maxnnz, 0, 0, 0).total >
                                     smem_limit() - 12288) {
        B.mode = mixed ? MODE_MIXED : MODE_FP64;
        if (B.mode == MODE_FP64 && !D.norm) D.norm = ar.alloc<double>(D.n);
        if (B.mode == MODE_MIXED && !D.vmix) {
            D.vmix = ar.alloc<float>(D.nnz);
            D.normf = ar.alloc<float>(D.n);
        }
        k_norms<<<grid1(D.n), 256, 0, st>>>(D.n, D.indptr, D.values, D.norm, D.vmix, D.normf, D.info);
        CK(cudaGetLastError());
        ++*launches;
    }
    B.dense = B.mode == MODE_MIXED && D.nnz == D.n * D.d;
    B.d_eff = (int)D.d;
    if (B.dense) {
        const int d_pad = (int)((D.d + 7) & ~7ll);
        B.dense_rows = ar.alloc<__nv_bfloat16>((size_t)D.n * d_pad);
        k_dense_bf16<<<(unsigned)D.n, 128, 0, st>>>(D.n, (int)D.d, d_pad, D.indptr, D.indices, D.vmix,
                                                    B.dense_rows);
        CK(cudaGetLastError());
        ++*launches;
        B.d_eff = d_pad;
    }
    B.ktab_len = B.mode == MODE_BINARY ? 2 * D.maxnnz + 1 : 0;
    B.smem = smo_batch_smem(B.mode, B.d_eff, B.ktab_len, D.maxnnz);
    if (B.smem > smem_limit() - 12288) {
        set_err("d = %lld exceeds the shared-memory target rows of the batched solver", (long long)D.d);
        throw Fail{SVM_ERR_UNSUPPORTED};
    }
}

// timed run of the batch kernel; returns device ms and fills results
float batch_run(const BatchPlan &P, const BatchArgs &A0, int lpr, int cs, int nclusters, int *next_job,
                cudaStream_t st, int *launches)
{
    BatchArgs A = A0;
    A.next_job = next_job;
    CK(cudaMemsetAsync(next_job, 0, sizeof(int), st));
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    CK(cudaEventRecord(e0, st));
    CK(launch_smo_batch(P.mode, lpr, P.dense, A, P.smem, cs, nclusters, st));
    ++*launches;
    CK(cudaEventRecord(e1, st));
    CK(cudaEventSynchronize(e1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ms;
}

int batch_clusters(const BatchPlan &P, int lpr, int cs)
{
    return smo_batch_max_clusters(P.mode, lpr, P.dense, P.smem, cs);
}

int train_batch_impl(const svm_csr *X, const svm_job *jobs, int32_t n_jobs, svm_batch_config *cfg,
                     svm_result *results, bool tune_only)
{
    auto t_start = std::chrono::steady_clock::now();
    if (!X || !jobs || !cfg || (!results && !tune_only)) ARG_FAIL("NULL argument");
    if (n_jobs < 1) ARG_FAIL("n_jobs must be >= 1");
    if (cfg->precision < SVM_FP64 || cfg->precision > SVM_MIXED_BF16_SIMT)
        ARG_FAIL("unknown precision %d", cfg->precision);
    if (cfg->cluster_size < 0 || cfg->cluster_size > 16 || (cfg->cluster_size & (cfg->cluster_size - 1)))
        ARG_FAIL("cluster_size must be 0 (autotune) or a power of two <= 16");
    cudaStream_t st = as_stream(cfg->stream);
    int launches = 0;
    Arena ar(st);
    BatchPlan P;
    batch_prepare(ar, X, cfg->precision, st, P, &launches);
    const DevCSR &D = P.D;

    // ---- concatenated job arrays
    std::vector<BatchJobDev> hj(n_jobs);
    std::vector<int64_t> offs(n_jobs);
    int64_t total = 0;
    for (int j = 0; j < n_jobs; ++j) {
        const svm_job &J = jobs[j];
        if (J.n_rows < 2) ARG_FAIL("job %d: need at least two rows", j);
        if (!J.rows && J.n_rows > D.n) ARG_FAIL("job %d: n_rows exceeds the matrix", j);
        if (!J.y || (!J.alpha_out && !tune_only)) ARG_FAIL("job %d: labels and alpha_out must not be NULL", j);
        if (!(J.C > 0) || !(J.gamma > 0) || !(J.tau > 0)) ARG_FAIL("job %d: C, gamma and tau must be > 0", j);
        if (J.n_rows >= INT32_MAX) ARG_FAIL("job %d: too many rows", j);
        std::memset(&hj[j], 0, sizeof(BatchJobDev));
        offs[j] = total;
        hj[j].nrows = (int32_t)J.n_rows;
        hj[j].C = J.C;
        hj[j].gamma = J.gamma;
        hj[j].tau = J.tau;
        hj[j].max_iter = J.max_iter > 0 ? J.max_iter : 100 * J.n_rows + 1000000;
        hj[j].xd = D.xd;
        total += J.n_rows;
    }
    int32_t *rows = ar.alloc<int32_t>(total);
    int8_t *ycat = ar.alloc<int8_t>(total);
    if (X->on_device) {
        for (int j = 0; j < n_jobs; ++j) {
            const svm_job &J = jobs[j];
            if (J.rows)
                CK(cudaMemcpyAsync(rows + offs[j], J.rows, 4 * J.n_rows, cudaMemcpyDeviceToDevice, st));
            else {
                k_iota<<<grid1(J.n_rows), 256, 0, st>>>(J.n_rows, rows + offs[j]);
                CK(cudaGetLastError());
                ++launches;
            }
            CK(cudaMemcpyAsync(ycat + offs[j], J.y, J.n_rows, cudaMemcpyDeviceToDevice, st));
        }
    } else {
        std::vector<int32_t> hr(total);
        std::vector<int8_t> hy(total);
        for (int j = 0; j < n_jobs; ++j) {
            const svm_job &J = jobs[j];
            for (int64_t r = 0; r < J.n_rows; ++r) hr[offs[j] + r] = J.rows ? J.rows[r] : (int32_t)r;
            std::memcpy(hy.data() + offs[j], J.y, J.n_rows);
        }
        CK(cudaMemcpyAsync(rows, hr.data(), 4 * total, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(ycat, hy.data(), total, cudaMemcpyHostToDevice, st));
        CK(cudaStreamSynchronize(st));
    }
    double *alpha = ar.alloc<double>(total);
    double *f = ar.alloc<double>(total);
    uint8_t *status = ar.alloc<uint8_t>(total);
    for (int j = 0; j < n_jobs; ++j) {
        BatchJobDev &J = hj[j];
        J.indptr = D.indptr;
        J.indices = D.indices;
        J.values = D.values;
        J.vmix = D.vmix;
        J.dmat = P.dense_rows;
        J.norm = D.norm;
        J.normf = D.normf;
        J.d = P.d_eff;
        J.dense = P.dense;
        J.rows = rows + offs[j];
        J.y = ycat + offs[j];
        J.alpha = alpha + offs[j];
        J.f = f + offs[j];
        J.status = status + offs[j];
    }
    BatchJobDev *djobs = ar.alloc<BatchJobDev>(n_jobs);
    CK(cudaMemcpyAsync(djobs, hj.data(), sizeof(BatchJobDev) * n_jobs, cudaMemcpyHostToDevice, st));
    int *bad = ar.alloc<int>(n_jobs);
    k_job_check<<<n_jobs, 256, 0, st>>>(n_jobs, djobs, D.n, bad);
    CK(cudaGetLastError());
    ++launches;
    std::vector<int> hbad(n_jobs);
    CK(cudaMemcpyAsync(hbad.data(), bad, sizeof(int) * n_jobs, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    for (int j = 0; j < n_jobs; ++j) {
        if (hbad[j] == 1) ARG_FAIL("job %d: row ids out of range or labels not +-1", j);
        if (hbad[j] == 2) ARG_FAIL("job %d: both classes must be present", j);
    }

    BatchResultDev *dres = ar.alloc<BatchResultDev>(n_jobs);
    int *next_job = ar.alloc<int>(1);
    BatchArgs A;
    std::memset(&A, 0, sizeof A);
    A.d = P.d_eff;
    A.njobs = n_jobs;
    A.jobs = djobs;
    A.results = dres;
    A.ktab_len = P.ktab_len;
    A.maxnnz = D.maxnnz;

    // ---- launch shape: given, or picked by timing candidates on a sample
    int cs = cfg->cluster_size, lpr = cfg->lanes_per_row;
    if (lpr > 0) {
        int l = 1;
        while (l < 32 && l < lpr) l <<= 1;
        lpr = l;
    }
    if (cs == 0 || lpr == 0) {
        const double avg = (double)D.nnz / (double)D.n;
        std::vector<int> lprs, css;
        if (lpr > 0) lprs = {lpr};
        else if (P.dense) lprs = {2, 4, 8, 16, 32};
        else if (avg <= 48) lprs = {1, 2, 4};
        else lprs = {2, 4, 8, 16};
        if (cs > 0) css = {cs};
        else css = {2, 4, 8, 16};
        // sample: up to 64 jobs, at most 300 steps each
        const int ns = std::min(n_jobs, 64);
        std::vector<BatchJobDev> sj(hj.begin(), hj.begin() + ns);
        for (auto &x : sj) x.max_iter = std::min<int64_t>(x.max_iter, 300);
        BatchJobDev *dsj = ar.alloc<BatchJobDev>(ns);
        CK(cudaMemcpyAsync(dsj, sj.data(), sizeof(BatchJobDev) * ns, cudaMemcpyHostToDevice, st));
        std::vector<BatchResultDev> sres(ns);
        BatchArgs S = A;
        S.jobs = dsj;
        S.njobs = ns;
        double best = -1.0;
        int best_cs = css[0], best_lpr = lprs[0];
        for (int c : css) {
            for (int l : lprs) {
                const int maxc = batch_clusters(P, l, c);
                if (maxc < 1) continue;
                const float ms = batch_run(P, S, l, c, std::min(maxc, ns), next_job, st, &launches);
                CK(cudaMemcpy(sres.data(), dres, sizeof(BatchResultDev) * ns, cudaMemcpyDeviceToHost));
                int64_t it = 0;
                for (auto &r : sres) it += r.iters;
                const double rate = (double)it / (double)std::max(ms, 1e-3f);
                if (rate > best) {
                    best = rate;
                    best_cs = c;
                    best_lpr = l;
                }
            }
        }
        if (best < 0) {
            set_err("no batched launch shape fits this device");
            throw Fail{SVM_ERR_UNSUPPORTED};
        }
        cs = best_cs;
        lpr = best_lpr;
        cfg->cluster_size = cs;
        cfg->lanes_per_row = lpr;
    }
    if (tune_only) return SVM_OK;
    const int maxc = batch_clusters(P, lpr, cs);
    if (maxc < 1) {
        set_err("cluster size %d does not fit this device", cs);
        throw Fail{SVM_ERR_UNSUPPORTED};
    }
    int ncl = std::min(maxc, n_jobs);
    if (cfg->clusters > 0) ncl = std::min(ncl, cfg->clusters);
    const float ms = batch_run(P, A, lpr, cs, ncl, next_job, st, &launches);
    std::vector<BatchResultDev> hres(n_jobs);
    CK(cudaMemcpyAsync(hres.data(), dres, sizeof(BatchResultDev) * n_jobs, cudaMemcpyDeviceToHost, st));
    if (X->on_device) {
        for (int j = 0; j < n_jobs; ++j)
            CK(cudaMemcpyAsync(jobs[j].alpha_out, alpha + offs[j], 8 * jobs[j].n_rows, cudaMemcpyDeviceToDevice,
                               st));
        CK(cudaStreamSynchronize(st));
    } else {
        std::vector<double> ha(total);
        CK(cudaMemcpyAsync(ha.data(), alpha, 8 * total, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        for (int j = 0; j < n_jobs; ++j)
            std::memcpy(jobs[j].alpha_out, ha.data() + offs[j], 8 * jobs[j].n_rows);
    }
    int64_t iters = 0;
    int rc = SVM_OK;
    for (int j = 0; j < n_jobs; ++j) {
        svm_result &R = results[j];
        R.b = hres[j].b;
        R.b_up = hres[j].b_up;
        R.b_low = hres[j].b_low;
        R.objective = hres[j].objective;
        R.iters = hres[j].iters;
        R.status = hres[j].status == 1 ? SVM_NOT_CONVERGED : SVM_OK;
        R.n_sv = hres[j].n_sv;
        iters += hres[j].iters;
        if (R.status != SVM_OK) rc = SVM_NOT_CONVERGED;
    }
    cfg->ms_kernel = ms;
    cfg->iters_total = iters;
    cfg->clusters_used = ncl;
    cfg->ms_total = elapsed_ms(t_start);
    g_launches += launches;
    return rc;
}


// ---------------------------------------------------------------------------
// Serving: continuous batching of training jobs that arrive over time
// ---------------------------------------------------------------------------

struct SrvJob {
    uint64_t ticket = 0;
    int state = 0;           // 0 queued, 1 on the device, 2 finished
    int slot = -1;
    bool cancelled = false;
    int64_t n = 0, d = 0, nnz = 0;
    std::vector<int64_t> indptr;
    std::vector<int32_t> indices;
    std::vector<float> values;
    std::vector<int8_t> y;
    double C = 1, gamma = 1, tau = 1e-3;
    int64_t max_iter = 0;
    size_t bytes = 0;
    void *mem = nullptr;
    double *alpha_d = nullptr;
    int rc = SVM_PENDING;
    std::string err;
    svm_result res{};
    std::vector<double> alpha;
    std::chrono::steady_clock::time_point t_submit, t_admit, t_done;
};

struct EngineCtl {
    unsigned tail;
    int shutdown;
    int pad[30];
};

struct Server {
    svm_server_config cfg{};
    int mode = MODE_MIXED;
    size_t used = 0;
    std::mutex mu;
    std::condition_variable cv;
    std::map<uint64_t, std::shared_ptr<SrvJob>> jobs;
    std::deque<uint64_t> queue;
    std::vector<int> free_slots;
    std::vector<std::shared_ptr<SrvJob>> running;
    uint64_t next_ticket = 1;
    std::thread worker;
    bool stop = false;
    int device = 0;
    cudaStream_t s_engine = nullptr, s_side = nullptr;
    EngineCtl *ctl_h = nullptr, *ctl_d = nullptr;
    int32_t *ring_h = nullptr, *ring_d = nullptr;
    BatchJobDev *slots_h = nullptr, *slots_d = nullptr;
    BatchResultDev *res_h = nullptr, *res_d = nullptr;
    int *done_h = nullptr, *done_d = nullptr;
    int *next_d = nullptr;
    IngestInfo *info_h = nullptr, *info_d = nullptr;
    size_t smem = 0;
    int nclusters = 0;
    int64_t engine_launches = 0;
    std::string fatal;
};

size_t srv_job_bytes(const SrvJob &J, int mode)
{
    auto a = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const bool dense = mode == MODE_MIXED && J.nnz == J.n * J.d;
    const size_t dpad = (size_t)((J.d + 7) & ~7ll);
    size_t b = a(8 * (J.n + 1)) + a(4 * J.nnz) + a(4 * J.nnz) + a(4 * J.n) + a(J.n) + a(8 * J.n) * 2 + a(J.n);
    if (mode == MODE_MIXED) b += a(4 * J.nnz) + a(4 * J.n);
    else b += a(8 * J.n);
    if (dense) b += a(2 * J.n * dpad);
    return b;
}

// one engine launch; the engine runs until shutdown or until idle
void srv_launch_engine(Server &S)
{
    BatchArgs A;
    std::memset(&A, 0, sizeof A);
    A.d = S.cfg.max_d;
    A.njobs = 0;
    A.jobs = S.slots_d;
    A.results = S.res_d;
    A.next_job = S.next_d;
    A.ktab_len = 0;
    A.maxnnz = S.cfg.max_d;
    A.ring = S.ring_d;
    A.ring_tail = &S.ctl_d->tail;
    A.ring_cap = S.cfg.max_slots;
    A.shutdown = &S.ctl_d->shutdown;
    A.done = S.done_d;
    A.idle_ns = 500ll * 1000 * 1000;
    CK(launch_smo_batch(S.mode, S.cfg.lanes_per_row, 0, A, S.smem, S.cfg.cluster_size, S.nclusters, S.s_engine));
    ++S.engine_launches;
    g_launches += 1;
}

// stage a queued job on the device and publish it to the engine (lock held)
void srv_admit(Server &S, const std::shared_ptr<SrvJob> &J)
{
    cudaStream_t st = S.s_side;
    const bool mixed = S.mode == MODE_MIXED;
    const bool dense = mixed && J->nnz == J->n * J->d;
    const int dpad = (int)((J->d + 7) & ~7ll);
    CK(cudaMallocAsync(&J->mem, J->bytes, st));
    unsigned char *p = static_cast<unsigned char *>(J->mem);
    auto take = [&](size_t x) {
        unsigned char *r = p;
        p += (x + 255) & ~(size_t)255;
        return r;
    };
    int64_t *indptr = reinterpret_cast<int64_t *>(take(8 * (J->n + 1)));
    int32_t *indices = reinterpret_cast<int32_t *>(take(4 * J->nnz));
    float *values = reinterpret_cast<float *>(take(4 * J->nnz));
    int32_t *rows = reinterpret_cast<int32_t *>(take(4 * J->n));
    int8_t *y = reinterpret_cast<int8_t *>(take(J->n));
    double *alpha = reinterpret_cast<double *>(take(8 * J->n));
    double *f = reinterpret_cast<double *>(take(8 * J->n));
    uint8_t *status = reinterpret_cast<uint8_t *>(take(J->n));
    float *vmix = nullptr, *normf = nullptr;
    double *norm = nullptr;
    __nv_bfloat16 *dmat = nullptr;
    if (mixed) {
        vmix = reinterpret_cast<float *>(take(4 * J->nnz));
        normf = reinterpret_cast<float *>(take(4 * J->n));
    } else {
        norm = reinterpret_cast<double *>(take(8 * J->n));
    }
    if (dense) dmat = reinterpret_cast<__nv_bfloat16 *>(take(2 * (size_t)J->n * dpad));
    CK(cudaMemcpyAsync(indptr, J->indptr.data(), 8 * (J->n + 1), cudaMemcpyHostToDevice, st));
    if (J->nnz) {
        CK(cudaMemcpyAsync(indices, J->indices.data(), 4 * J->nnz, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(values, J->values.data(), 4 * J->nnz, cudaMemcpyHostToDevice, st));
    }
    CK(cudaMemcpyAsync(y, J->y.data(), J->n, cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(S.info_d, 0, sizeof(IngestInfo), st));
    k_validate<<<grid1(J->n), 256, 0, st>>>(J->n, J->d, indptr, indices, values, y, S.info_d);
    k_norms<<<grid1(J->n), 256, 0, st>>>(J->n, indptr, values, norm, vmix, normf, S.info_d);
    k_iota<<<grid1(J->n), 256, 0, st>>>(J->n, rows);
    if (dense) k_dense_bf16<<<(unsigned)J->n, 128, 0, st>>>(J->n, (int)J->d, dpad, indptr, indices, vmix, dmat);
    CK(cudaGetLastError());
    g_launches += dense ? 4 : 3;
    CK(cudaMemcpyAsync(S.info_h, S.info_d, sizeof(IngestInfo), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    const IngestInfo &h = *S.info_h;
    std::string bad;
    if (h.bad_indptr) bad = "indptr is not non-decreasing from 0";
    else if (h.bad_index) bad = "column indices must be strictly increasing within a row and < d";
    else if (h.nonfinite) bad = "values must be finite";
    else if (h.bad_y) bad = "labels must be +1 or -1";
    else if (h.npos == 0 || (int64_t)h.npos == J->n) bad = "both classes must be present";
    if (!bad.empty()) {
        CK(cudaFreeAsync(J->mem, st));
        J->mem = nullptr;
        J->rc = SVM_ERR_ARG;
        J->err = bad;
        J->state = 2;
        J->t_done = std::chrono::steady_clock::now();
        S.used -= J->bytes;
        return;
    }
    const int slot = S.free_slots.back();
    S.free_slots.pop_back();
    J->slot = slot;
    J->alpha_d = alpha;
    BatchJobDev &D = S.slots_h[slot];
    std::memset(&D, 0, sizeof D);
    D.indptr = indptr;
    D.indices = indices;
    D.values = values;
    D.vmix = vmix;
    D.dmat = dmat;
    D.norm = norm;
    D.normf = normf;
    D.rows = rows;
    D.y = y;
    D.alpha = alpha;
    D.f = f;
    D.status = status;
    D.nrows = (int32_t)J->n;
    D.d = dense ? dpad : (int32_t)J->d;
    D.dense = dense ? 1 : 0;
    D.C = J->C;
    D.gamma = J->gamma;
    D.tau = J->tau;
    D.max_iter = J->max_iter > 0 ? J->max_iter : 100 * J->n + 1000000;
    D.xd = xd_of_info(h, values);
    __atomic_store_n(&S.done_h[slot], 0, __ATOMIC_RELAXED);
    const unsigned tail = __atomic_load_n(&S.ctl_h->tail, __ATOMIC_RELAXED);
    S.ring_h[tail % (unsigned)S.cfg.max_slots] = slot;
    __atomic_store_n(&S.ctl_h->tail, tail + 1, __ATOMIC_RELEASE);   // publishes descriptor and ring entry
    J->state = 1;
    J->t_admit = std::chrono::steady_clock::now();
    S.running.push_back(J);
}

// collect a finished job (lock held)
void srv_finish(Server &S, const std::shared_ptr<SrvJob> &J)
{
    const BatchResultDev &R = S.res_h[J->slot];
    J->res.b = R.b;
    J->res.b_up = R.b_up;
    J->res.b_low = R.b_low;
    J->res.objective = R.objective;
    J->res.iters = R.iters;
    J->res.status = R.status == 1 ? SVM_NOT_CONVERGED : SVM_OK;
    J->res.n_sv = R.n_sv;
    J->alpha.resize(J->n);
    CK(cudaMemcpyAsync(J->alpha.data(), J->alpha_d, 8 * J->n, cudaMemcpyDeviceToHost, S.s_side));
    CK(cudaFreeAsync(J->mem, S.s_side));
    CK(cudaStreamSynchronize(S.s_side));
    J->mem = nullptr;
    J->rc = J->cancelled ? SVM_ERR_CANCELLED : J->res.status;
    J->state = 2;
    J->t_done = std::chrono::steady_clock::now();
    S.used -= J->bytes;
    S.free_slots.push_back(J->slot);
}

void srv_loop(Server *S)
{
    CK_NOTHROW(cudaSetDevice(S->device));
    std::unique_lock<std::mutex> lk(S->mu);
    while (!S->stop) {
        try {
            // finished jobs
            for (size_t k = 0; k < S->running.size();) {
                auto &J = S->running[k];
                if (__atomic_load_n(&S->done_h[J->slot], __ATOMIC_ACQUIRE)) {
                    srv_finish(*S, J);
                    S->running.erase(S->running.begin() + k);
                    S->cv.notify_all();
                } else {
                    ++k;
                }
            }
            // admission: first come, first served while a slot and budget are free
            while (!S->queue.empty() && !S->free_slots.empty()) {
                auto it = S->jobs.find(S->queue.front());
                if (it == S->jobs.end() || it->second->state != 0) {
                    S->queue.pop_front();
                    continue;
                }
                auto J = it->second;
                if (S->used + J->bytes > S->cfg.budget_bytes) break;
                S->queue.pop_front();
                S->used += J->bytes;
                srv_admit(*S, J);
                if (J->state == 2) S->cv.notify_all();
            }
            // the engine leaves when idle: start it again while work is out
            if (!S->running.empty() && cudaStreamQuery(S->s_engine) == cudaSuccess) srv_launch_engine(*S);
        } catch (const Fail &) {
            S->fatal = g_err;
            for (auto &J : S->running) {
                J->rc = SVM_ERR_CUDA;
                J->err = S->fatal;
                J->state = 2;
            }
            S->running.clear();
            S->cv.notify_all();
        }
        S->cv.wait_for(lk, std::chrono::microseconds(S->running.empty() && S->queue.empty() ? 2000 : 50));
    }
}

double ms_between(std::chrono::steady_clock::time_point a, std::chrono::steady_clock::time_point b)
{
    return std::chrono::duration<double, std::milli>(b - a).count();
}

// ---------------------------------------------------------------------------
// Fixed-workspace training: a variant of the plain (no shrinking) FP64 solve
// that allocates nothing. Some callers cannot allocate device memory during
// a call: code running inside a memory-capped or externally managed pool, a
// real-time loop that must not block on the allocator, or a host that
// reserved the whole device up front. For them every piece of scratch the
// solve needs lives in one file-scope device array, placed in a GPU's memory
// when this file's code is first loaded there (with lazy module loading, the
// first call that runs device work on that GPU); inputs and outputs are the
// caller's device buffers.
// ---------------------------------------------------------------------------
constexpr int64_t kFixedMaxRows = 131072;            // largest n accepted
constexpr int kFixedMaxRowNnz = 4096;                // longest row accepted
constexpr size_t kFixedScratchBytes = (size_t)4 << 20;   // 4 MiB per device

static __device__ __align__(256) unsigned char g_fixed_scratch[kFixedScratchBytes];

// Device address of g_fixed_scratch, looked up once per device.
constexpr int kMaxDevices = 64;
std::mutex g_fixed_mu;
void *g_fixed_addr[kMaxDevices] = {};

void *fixed_scratch_address()
{
    int dev = 0;
    CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        set_err("device index %d out of range for the fixed workspace", dev);
        throw Fail{SVM_ERR_UNSUPPORTED};
    }
    std::lock_guard<std::mutex> lk(g_fixed_mu);
    if (!g_fixed_addr[dev]) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_fixed_scratch);
        if (e != cudaSuccess || !ptr) {
            set_err("cudaGetSymbolAddress of the fixed workspace failed: %s", cudaGetErrorString(e));
            throw Fail{SVM_ERR_CUDA};
        }
        g_fixed_addr[dev] = ptr;
    }
    return g_fixed_addr[dev];
}

// Carves aligned pieces out of the fixed workspace.
struct FixedCarve {
    unsigned char *base;
    size_t used = 0;
    template <class T>
    T *take(size_t count)
    {
        size_t off = (used + 255) & ~(size_t)255;
        size_t bytes = (count ? count : 1) * sizeof(T);
        if (off + bytes > kFixedScratchBytes) {
            set_err("problem needs more than the %zu-byte fixed workspace", kFixedScratchBytes);
            throw Fail{SVM_ERR_UNSUPPORTED};
        }
        used = off + bytes;
        return reinterpret_cast<T *>(base + off);
    }
};

int train_fixed_impl(const svm_csr *X, const int8_t *y, const svm_params *P, double *alpha_out,
                     double *b_out, int64_t *iters_out)
{
    if (P && P->alpha0) ARG_FAIL("alpha0 (warm start) is not taken by the fixed-workspace solve");
    if (!X || !P || !y || !alpha_out || !b_out) ARG_FAIL("NULL argument");
    if (!X->on_device) ARG_FAIL("the fixed-workspace call takes device buffers only (on_device = 1)");
    if (!(P->C > 0) || !std::isfinite(P->C)) ARG_FAIL("C must be > 0");
    if (!(P->gamma > 0) || !std::isfinite(P->gamma)) ARG_FAIL("gamma must be > 0");
    if (!(P->tau > 0) || !std::isfinite(P->tau)) ARG_FAIL("tau must be > 0");
    if (P->precision != SVM_FP64) ARG_FAIL("the fixed-workspace call supports SVM_FP64 only");
    if (P->kernel != SVM_KERNEL_RBF) ARG_FAIL("the fixed-workspace call supports the RBF kernel only");
    if (P->tie_break != 0) ARG_FAIL("only the lowest-index tie-break (0) is implemented");
    if (X->n < 2 || X->d < 1) ARG_FAIL("need n >= 2 and d >= 1");
    if (X->d >= (int64_t)INT32_MAX) ARG_FAIL("d must be < 2^31");
    if (X->n > kFixedMaxRows) {
        set_err("n = %lld exceeds the fixed workspace limit of %lld rows", (long long)X->n,
                (long long)kFixedMaxRows);
        throw Fail{SVM_ERR_UNSUPPORTED};
    }
    if (!X->indptr || !X->indices) ARG_FAIL("indptr/indices must not be NULL");
    cudaStream_t st = as_stream(P->stream);
    FixedCarve W{static_cast<unsigned char *>(fixed_scratch_address())};
    const int64_t n = X->n;
    int launches = 0;

    // ingest checks (device buffers are read in place)
    IngestInfo *info = W.take<IngestInfo>(1);
    CK(cudaMemsetAsync(info, 0, sizeof(IngestInfo), st));
    k_validate<<<grid1(n), 256, 0, st>>>(n, X->d, X->indptr, X->indices, X->values, y, info);
    CK(cudaGetLastError());
    ++launches;
    IngestInfo h;
    int64_t nnz = 0;
    CK(cudaMemcpyAsync(&h, info, sizeof h, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&nnz, X->indptr + n, sizeof nnz, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (h.bad_indptr) ARG_FAIL("indptr is not non-decreasing from 0");
    if (h.bad_index) ARG_FAIL("column indices must be strictly increasing within a row and < d");
    if (h.nonfinite) ARG_FAIL("values must be finite");
    if (h.bad_y) ARG_FAIL("labels must be +1 or -1");
    if (h.npos == 0 || (int64_t)h.npos == n) ARG_FAIL("both classes must be present");
    if (h.maxnnz > kFixedMaxRowNnz) {
        set_err("a row has %d entries; the fixed workspace accepts at most %d", h.maxnnz, kFixedMaxRowNnz);
        throw Fail{SVM_ERR_UNSUPPORTED};
    }
    // (the larger of the two modes' static shared memory: the mode is decided below)
    const size_t lim_dyn = smem_limit() - std::max(smo_static_smem(MODE_BINARY), smo_static_smem(MODE_FP64)) - 1024;
    // binary input whose distance tables do not fit in shared memory takes
    // the generic FP64 row pass with norms, as svm_train does
    bool binary = !h.not_binary;
    const int ktab_len = 2 * h.maxnnz + 1;
    if (binary && smo_layout(MODE_BINARY, (int)X->d, ktab_len, h.maxnnz, 0, 0, 0).total > lim_dyn) {
        if (!X->values) {
            set_err("d = %lld is too large for the binary tables and values is NULL (the FP64 row "
                    "pass of the fixed-workspace call needs explicit values)", (long long)X->d);
            throw Fail{SVM_ERR_UNSUPPORTED};
        }
        binary = false;
    }
    const int mode = binary ? MODE_BINARY : MODE_FP64;
    double *norm = nullptr, *ktab = nullptr;
    if (binary) {
        ktab = W.take<double>(3 * (size_t)ktab_len);
        k_ktab<<<grid1(ktab_len), 256, 0, st>>>(P->gamma, ktab_len, ktab);
    } else {
        norm = W.take<double>(n);
        k_norms<<<grid1(n), 256, 0, st>>>(n, X->indptr, X->values, norm, nullptr, nullptr, info);
    }
    CK(cudaGetLastError());
    ++launches;

    // launch shape: the same rules as svm_train, rows streamed from global
    const double avg = (double)nnz / (double)n;
    int lpr = 1;
    while (lpr < 32 && lpr * 32 < avg) lpr <<= 1;
    const int sms = device_sms();
    int G = (int)std::min<int64_t>(sms, std::max<int64_t>(1, (n + 15) / 16));
    if (G > 256) G = 256;
    const SmoLayout L0 = smo_layout(mode, (int)X->d, binary ? ktab_len : 0, h.maxnnz, 0, 0, 0);
    if (L0.total > lim_dyn) {
        set_err("d = %lld exceeds the shared-memory target rows of this mode", (long long)X->d);
        throw Fail{SVM_ERR_UNSUPPORTED};
    }
    int cs = 1;
    if (G >= 16) {
        const int maxc = smo_max_clusters(mode, lpr, 0, L0.total, 8);
        if (maxc >= 2) {
            cs = 8;
            G = 8 * std::min(maxc, G / 8);
        }
    }

    // solver state: alpha lives in the caller's output buffer
    double *f = W.take<double>(n);
    uint8_t *status = W.take<uint8_t>(n);
    int32_t *act = W.take<int32_t>(n);
    int32_t *seg_cnt = W.take<int32_t>(G);
    void *cand = W.take<unsigned char>(smo_cand_slots(G) * smo_cand_bytes());
    unsigned *seq = W.take<unsigned>(smo_seq_words(G));
    SmoCtrl *ctrl = W.take<SmoCtrl>(1);
    const int nbf = (int)std::min<int64_t>(1024, std::max<int64_t>(1, (n + 4095) / 4096));
    FinishPart *parts = W.take<FinishPart>(nbf);
    FinishPart *tot = W.take<FinishPart>(1);
    k_init<<<grid1(n), 256, 0, st>>>(n, y, alpha_out, f, status);
    k_reset_active<<<G, 256, 0, st>>>(n, G, act, seg_cnt);
    CK(cudaGetLastError());
    launches += 2;

    SmoCtrl hc;
    std::memset(&hc, 0, sizeof hc);
    hc.active = n;
    hc.i_up = hc.i_low = -1;
    SmoArgs A;
    std::memset(&A, 0, sizeof A);
    A.n = n;
    A.d = (int32_t)X->d;
    A.G = G;
    A.indptr = X->indptr;
    A.indices = X->indices;
    A.values = X->values;
    A.y = y;
    A.norm = norm;
    A.alpha = alpha_out;
    A.f = f;
    A.status = status;
    A.act = act;
    A.seg_cnt = seg_cnt;
    A.cand = cand;
    A.seq = seq;
    A.ctrl = ctrl;
    A.ktab = ktab;
    A.ktab_len = ktab_len;
    A.maxnnz = h.maxnnz;
    A.xd = xd_of_info(h, X->values);
    A.resident = 0;
    A.C = P->C;
    A.gamma = P->gamma;
    A.thr = 2.0 * P->tau;
    A.iter_limit = P->max_iter > 0 ? P->max_iter : 100 * n + 1000000;
    A.h = 0;
    A.select_only = 1;
    A.wss2 = (P->flags & SVM_FLAG_WSS2) != 0;
    A.timeout_ns = 10ll * 1000 * 1000 * 1000;
    // every call starts from a zeroed exchange area and a fresh control block
    CK(cudaMemcpyAsync(ctrl, &hc, sizeof hc, cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(seq, 0, sizeof(unsigned) * smo_seq_words(G), st));
    CK(cudaMemsetAsync(cand, 0, smo_cand_slots(G) * smo_cand_bytes(), st));
    CK(launch_smo_persistent(mode, lpr, A, L0.total, st, cs));
    ++launches;
    CK(cudaMemcpyAsync(&hc, ctrl, sizeof hc, cudaMemcpyDeviceToHost, st));
    k_finish_part<<<nbf, kCT, 0, st>>>(n, P->C, alpha_out, f, status, parts);
    k_finish_total<<<1, 32, 0, st>>>(parts, nbf, tot);
    CK(cudaGetLastError());
    launches += 2;
    FinishPart fp;
    CK(cudaMemcpyAsync(&fp, tot, sizeof fp, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    g_launches += launches;
    if (hc.err) {
        set_err("a grid-wide wait in the SMO kernel exceeded its time limit");
        throw Fail{SVM_ERR_TIMEOUT};
    }
    *b_out = fp.n0 > 0 ? fp.sum_f0 / (double)fp.n0 : 0.5 * (hc.b_up + hc.b_low);
    if (iters_out) *iters_out = hc.iter;
    return hc.exit_reason == 1 ? SVM_NOT_CONVERGED : SVM_OK;
}

}  // namespace

extern "C" {

int svm_train(const svm_csr *X, const int8_t *y, const svm_params *params,
              const svm_shrink_policy *policy, double *alpha_out, double *b_out,
              int64_t *iters_out, svm_stats *stats)
{
    g_err.clear();
    try {
        if (!X) ARG_FAIL("X is NULL");
        return train_impl(X, y, params, policy, alpha_out, b_out, iters_out, stats);
    } catch (const Fail &f) {
        return f.code;
    } catch (...) {
        set_err("unexpected host exception");
        return SVM_ERR_CUDA;
    }
}

int svm_decision(const svm_csr *X, const int8_t *y, const double *alpha, double b, double gamma,
                 const svm_csr *Z, int32_t precision, void *stream, double *out)
{
    g_err.clear();
    try {
        svm_kernel K;
        K.kind = SVM_KERNEL_RBF;
        K.degree = 3;
        K.gamma = gamma;
        K.coef0 = 0.0;
        return decision_impl(X, y, alpha, b, K, Z, precision, stream, out);
    } catch (const Fail &f) {
        return f.code;
    } catch (...) {
        set_err("unexpected host exception");
        return SVM_ERR_CUDA;
    }
}

int svm_decision_kernel(const svm_csr *X, const int8_t *y, const double *alpha, double b,
                        const svm_kernel *kernel, const svm_csr *Z, int32_t precision, void *stream,
                        double *out)
{
    g_err.clear();
    try {
        if (!kernel) ARG_FAIL("kernel is NULL");
        return decision_impl(X, y, alpha, b, *kernel, Z, precision, stream, out);
    } catch (const Fail &f) {
        return f.code;
    } catch (...) {
        set_err("unexpected host exception");
        return SVM_ERR_CUDA;
    }
}

struct svm_model {
    ModelState *impl;
};

int svm_model_create(const svm_csr *X, const int8_t *y, const double *alpha, double b, const svm_kernel *kernel,
                     int32_t precision, void *stream, svm_model **out)
{
    g_err.clear();
    try {
        if (!out) ARG_FAIL("out is NULL");
        *out = nullptr;
        if (!kernel) ARG_FAIL("kernel is NULL");
        ModelState *M = model_create_impl(X, y, alpha, b, *kernel, precision, stream);
        svm_model *h = new (std::nothrow) svm_model;
        if (!h) {
            model_free_impl(M);
            set_err("host allocation failed");
            return SVM_ERR_OOM;
        }
        h->impl = M;
        *out = h;
        return SVM_OK;
    } catch (const Fail &f) {
        return f.code;
    } catch (...) {
        set_err("unexpected host exception");
        return SVM_ERR_CUDA;
    }
}

int svm_model_decision(const svm_model *model, const svm_csr *Z, void *stream, double *out)
{
    g_err.clear();
    try {
        if (!model || !model->impl || !Z || !out) ARG_FAIL("NULL argument");
        const ModelState &M = *model->impl;
        if (Z->d != M.sv.d) ARG_FAIL("Z->d (%lld) must equal the model's d (%lld)", (long long)Z->d, (long long)M.sv.d);
        int dev = 0;
        CK(cudaGetDevice(&dev));
        if (dev != M.device) ARG_FAIL("the model lives on device %d, the current device is %d", M.device, dev);
        if (Z->n == 0) return SVM_OK;
        cudaStream_t st = as_stream(stream);
        int launches = 0;
        Arena ar(st);
        decision_eval(ar, M.sv, M.list, M.coef, M.nsv, M.b, M.K, Z, M.precision, st, out, &launches);
        g_launches += launches;
        return SVM_OK;
    } catch (const Fail &f) {
        return f.code;
    } catch (...) {
        set_err("unexpected host exception");
        return SVM_ERR_CUDA;
    }
}

int svm_model_info(const svm_model *model, int64_t *n_sv, int64_t *d, double *b)
{
    g_err.clear();
    if (!model || !model->impl) {
        set_err("model is NULL");
        return SVM_ERR_ARG;
    }
    if (n_sv) *n_sv = model->impl->nsv;
    if (d) *d = model->impl->sv.d;
    if (b) *b = model->impl->b;
    return SVM_OK;
}

int svm_model_free(svm_model *model)
{
    g_err.clear();
    if (!model) return SVM_OK;
    model_free_impl(model->impl);
    delete model;
    return SVM_OK;
}

const char *svm_last_error(void) { return g_err.c_str(); }

int64_t svm_kernel_launches(void) { return (int64_t)g_launches.load(); }

int svm_diag_sfu_rate(double *ex2_per_s, void *stream)
{
    g_err.clear();
    try {
        if (!ex2_per_s) ARG_FAIL("NULL argument");
        CK(measure_sfu_ex2(ex2_per_s, as_stream(stream)));
        g_launches += 2;
        return SVM_OK;
    } catch (const Fail &f) {
        return f.code;
    } catch (...) {
        set_err("unexpected host exception");
        return SVM_ERR_CUDA;
    }
}

int svm_diag_wait_timeout(int64_t limit_ns, void *stream)
{
    g_err.clear();
    try {
        if (limit_ns < 1000000 || limit_ns > 5000000000ll) ARG_FAIL("limit_ns must be in [1e6, 5e9]");
        cudaStream_t st = as_stream(stream);
        Arena ar(st);
        int *dev = ar.alloc<int>(2);   // [0] error flag of other CTAs (0), [1] gave up
        CK(cudaMemsetAsync(dev, 0, 2 * sizeof(int), st));
        CK(launch_diag_wait(limit_ns, dev, dev + 1, st));
        g_launches += 1;
        int gave_up = 0;
        CK(cudaMemcpyAsync(&gave_up, dev + 1, sizeof gave_up, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (gave_up) {
            set_err("a device-side wait exceeded its limit of %lld ns", (long long)limit_ns);
            return SVM_ERR_TIMEOUT;
        }
        return SVM_OK;
    } catch (const Fail &f) {
        return f.code;
    } catch (...) {
        set_err("unexpected host exception");
        return SVM_ERR_CUDA;
    }
}

int svm_train_batch(const svm_csr *X, const svm_job *jobs, int32_t n_jobs, svm_batch_config *config,
                    svm_result *results)
{
    g_err.clear();
    try {
        return train_batch_impl(X, jobs, n_jobs, config, results, false);
    } catch (const Fail &f) {
        return f.code;
    } catch (...) {
        set_err("unexpected host exception");
        return SVM_ERR_CUDA;
    }
}

int svm_batch_autotune(const svm_csr *X, const svm_job *jobs, int32_t n_jobs, svm_batch_config *config)
{
    g_err.clear();
    try {
        return train_batch_impl(X, jobs, n_jobs, config, nullptr, true);
    } catch (const Fail &f) {
        return f.code;
    } catch (...) {
        set_err("unexpected host exception");
        return SVM_ERR_CUDA;
    }
}


struct svm_server {
    Server impl;
};

int svm_server_create(const svm_server_config *config, svm_server **out)
{
    g_err.clear();
    try {
        if (!config || !out) ARG_FAIL("NULL argument");
        svm_server_config c = *config;
        if (c.budget_bytes == 0) ARG_FAIL("budget_bytes must be > 0");
        if (c.max_slots <= 0) c.max_slots = 64;
        if (c.max_slots > 1024) ARG_FAIL("max_slots must be <= 1024");
        if (c.precision != SVM_FP64 && c.precision != SVM_MIXED_BF16 && c.precision != SVM_MIXED_BF16_SIMT)
            ARG_FAIL("unknown precision %d", c.precision);
        if (c.cluster_size <= 0) c.cluster_size = 16;
        if (c.cluster_size > 16 || (c.cluster_size & (c.cluster_size - 1))) ARG_FAIL("cluster_size must be a power of two <= 16");
        if (c.lanes_per_row <= 0) c.lanes_per_row = 2;
        {
            int l = 1;
            while (l < 32 && l < c.lanes_per_row) l <<= 1;
            c.lanes_per_row = l;
        }
        if (c.max_d <= 0) c.max_d = 2048;
        c.max_d = (c.max_d + 7) & ~7;
        auto S = std::make_unique<svm_server>();
        Server &V = S->impl;
        V.cfg = c;
        V.mode = c.precision == SVM_FP64 ? MODE_FP64 : MODE_MIXED;
        V.smem = smo_batch_smem(V.mode, c.max_d, 0, c.max_d);
        if (V.smem > smem_limit() - 12288) ARG_FAIL("max_d = %d does not fit the engine's shared memory", c.max_d);
        V.nclusters = smo_batch_max_clusters(V.mode, c.lanes_per_row, 0, V.smem, c.cluster_size);
        if (V.nclusters < 1) ARG_FAIL("cluster_size %d does not fit this device", c.cluster_size);
        CK(cudaGetDevice(&V.device));
        CK(cudaStreamCreateWithFlags(&V.s_engine, cudaStreamNonBlocking));
        CK(cudaStreamCreateWithFlags(&V.s_side, cudaStreamNonBlocking));
        auto mapped = [&](auto **h, auto **d, size_t bytes) {
            void *p = nullptr;
            CK(cudaHostAlloc(&p, bytes, cudaHostAllocMapped));
            std::memset(p, 0, bytes);
            void *q = nullptr;
            CK(cudaHostGetDevicePointer(&q, p, 0));
            *h = static_cast<std::remove_reference_t<decltype(**h)> *>(p);
            *d = static_cast<std::remove_reference_t<decltype(**d)> *>(q);
        };
        mapped(&V.ctl_h, &V.ctl_d, sizeof(EngineCtl));
        mapped(&V.ring_h, &V.ring_d, sizeof(int32_t) * c.max_slots);
        mapped(&V.slots_h, &V.slots_d, sizeof(BatchJobDev) * c.max_slots);
        mapped(&V.res_h, &V.res_d, sizeof(BatchResultDev) * c.max_slots);
        mapped(&V.done_h, &V.done_d, sizeof(int) * c.max_slots);
        mapped(&V.info_h, &V.info_d, sizeof(IngestInfo));
        // the ingest check writes into device memory, then copies to the mapped record
        void *infod = nullptr;
        CK(cudaMalloc(&infod, sizeof(IngestInfo)));
        V.info_d = static_cast<IngestInfo *>(infod);
        void *nd = nullptr;
        CK(cudaMalloc(&nd, sizeof(int)));
        CK(cudaMemset(nd, 0, sizeof(int)));
        V.next_d = static_cast<int *>(nd);
        for (int k = c.max_slots - 1; k >= 0; --k) V.free_slots.push_back(k);
        V.worker = std::thread(srv_loop, &V);
        *out = S.release();
        return SVM_OK;
    } catch (const Fail &f) {
        return f.code;
    } catch (...) {
        set_err("unexpected host exception");
        return SVM_ERR_CUDA;
    }
}

int svm_server_submit(svm_server *srv, const svm_csr *X, const int8_t *y, const svm_params *params,
                      uint64_t *ticket)
{
    g_err.clear();
    try {
        if (!srv || !X || !y || !params || !ticket) ARG_FAIL("NULL argument");
        if (X->on_device) ARG_FAIL("svm_server_submit takes host buffers (they are copied)");
        if (X->n < 2 || X->d < 1) ARG_FAIL("need n >= 2 and d >= 1");
        if (X->n >= INT32_MAX) ARG_FAIL("n must be < 2^31");
        if (!(params->C > 0) || !(params->gamma > 0) || !(params->tau > 0)) ARG_FAIL("C, gamma and tau must be > 0");
        Server &V = srv->impl;
        if (X->d > V.cfg.max_d) {
            set_err("d = %lld exceeds the server's max_d = %d", (long long)X->d, V.cfg.max_d);
            throw Fail{SVM_ERR_UNSUPPORTED};
        }
        auto J = std::make_shared<SrvJob>();
        J->n = X->n;
        J->d = X->d;
        J->nnz = X->indptr[X->n];
        if (J->nnz < 0) ARG_FAIL("indptr[n] < 0");
        J->indptr.assign(X->indptr, X->indptr + X->n + 1);
        J->indices.assign(X->indices, X->indices + J->nnz);
        if (X->values) J->values.assign(X->values, X->values + J->nnz);
        else J->values.assign(J->nnz, 1.0f);
        J->y.assign(y, y + X->n);
        J->C = params->C;
        J->gamma = params->gamma;
        J->tau = params->tau;
        J->max_iter = params->max_iter;
        J->bytes = srv_job_bytes(*J, V.mode);
        if (J->bytes > V.cfg.budget_bytes) {
            set_err("job needs %zu bytes of device memory; the budget is %zu", J->bytes, V.cfg.budget_bytes);
            throw Fail{SVM_ERR_BUDGET};
        }
        J->t_submit = std::chrono::steady_clock::now();
        {
            std::lock_guard<std::mutex> lk(V.mu);
            if (!V.fatal.empty()) {
                set_err("server stopped: %s", V.fatal.c_str());
                throw Fail{SVM_ERR_CUDA};
            }
            J->ticket = V.next_ticket++;
            V.jobs[J->ticket] = J;
            V.queue.push_back(J->ticket);
        }
        V.cv.notify_all();
        *ticket = J->ticket;
        return SVM_OK;
    } catch (const Fail &f) {
        return f.code;
    } catch (...) {
        set_err("unexpected host exception");
        return SVM_ERR_CUDA;
    }
}

static int srv_take(Server &V, uint64_t ticket, svm_result *res, double *alpha_out, svm_server_times *times)
{
    auto it = V.jobs.find(ticket);
    if (it == V.jobs.end()) ARG_FAIL("unknown ticket %llu", (unsigned long long)ticket);
    auto J = it->second;
    if (J->state != 2) return SVM_PENDING;
    if (res) *res = J->res;
    if (alpha_out && !J->alpha.empty()) std::memcpy(alpha_out, J->alpha.data(), 8 * J->n);
    if (times) {
        times->submit_to_admit_ms = J->t_admit.time_since_epoch().count() ? ms_between(J->t_submit, J->t_admit) : 0.0;
        times->admit_to_done_ms = J->t_admit.time_since_epoch().count() ? ms_between(J->t_admit, J->t_done) : 0.0;
        times->submit_to_done_ms = ms_between(J->t_submit, J->t_done);
    }
    const int rc = J->rc;
    if (rc < 0) set_err("%s", J->err.empty() ? "job failed" : J->err.c_str());
    V.jobs.erase(it);
    return rc;
}

int svm_server_poll(svm_server *srv, uint64_t ticket, svm_result *res, double *alpha_out,
                    svm_server_times *times)
{
    g_err.clear();
    try {
        if (!srv) ARG_FAIL("NULL server");
        Server &V = srv->impl;
        std::lock_guard<std::mutex> lk(V.mu);
        return srv_take(V, ticket, res, alpha_out, times);
    } catch (const Fail &f) {
        return f.code;
    } catch (...) {
        set_err("unexpected host exception");
        return SVM_ERR_CUDA;
    }
}

int svm_server_wait(svm_server *srv, uint64_t ticket, double timeout_s, svm_result *res, double *alpha_out,
                    svm_server_times *times)
{
    g_err.clear();
    try {
        if (!srv) ARG_FAIL("NULL server");
        Server &V = srv->impl;
        std::unique_lock<std::mutex> lk(V.mu);
        auto it = V.jobs.find(ticket);
        if (it == V.jobs.end()) ARG_FAIL("unknown ticket %llu", (unsigned long long)ticket);
        auto J = it->second;
        const auto until = std::chrono::steady_clock::now() +
                           std::chrono::microseconds((int64_t)(std::max(0.0, timeout_s) * 1e6));
        while (J->state != 2) {
            if (V.cv.wait_until(lk, until) == std::cv_status::timeout && J->state != 2) return SVM_PENDING;
        }
        return srv_take(V, ticket, res, alpha_out, times);
    } catch (const Fail &f) {
        return f.code;
    } catch (...) {
        set_err("unexpected host exception");
        return SVM_ERR_CUDA;
    }
}

int svm_server_cancel(svm_server *srv, uint64_t ticket)
{
    g_err.clear();
    try {
        if (!srv) ARG_FAIL("NULL server");
        Server &V = srv->impl;
        std::lock_guard<std::mutex> lk(V.mu);
        auto it = V.jobs.find(ticket);
        if (it == V.jobs.end()) ARG_FAIL("unknown ticket %llu", (unsigned long long)ticket);
        auto J = it->second;
        if (J->state == 0) {
            J->state = 2;
            J->rc = SVM_ERR_CANCELLED;
            J->err = "cancelled";
            J->t_done = std::chrono::steady_clock::now();
            V.cv.notify_all();
        } else if (J->state == 1) {
            J->cancelled = true;
        }
        return SVM_OK;
    } catch (const Fail &f) {
        return f.code;
    } catch (...) {
        set_err("unexpected host exception");
        return SVM_ERR_CUDA;
    }
}

int svm_server_stats(svm_server *srv, svm_server_info *info)
{
    g_err.clear();
    if (!srv || !info) {
        set_err("NULL argument");
        return SVM_ERR_ARG;
    }
    Server &V = srv->impl;
    std::lock_guard<std::mutex> lk(V.mu);
    info->bytes_in_use = V.used;
    info->budget_bytes = V.cfg.budget_bytes;
    info->queued = 0;
    for (auto t : V.queue) {
        auto it = V.jobs.find(t);
        if (it != V.jobs.end() && it->second->state == 0) ++info->queued;
    }
    info->running = (int32_t)V.running.size();
    info->clusters = V.nclusters;
    info->cluster_size = V.cfg.cluster_size;
    info->engine_launches = V.engine_launches;
    return SVM_OK;
}

int svm_server_destroy(svm_server *srv)
{
    g_err.clear();
    if (!srv) return SVM_OK;
    Server &V = srv->impl;
    {
        std::lock_guard<std::mutex> lk(V.mu);
        V.stop = true;
    }
    V.cv.notify_all();
    if (V.worker.joinable()) V.worker.join();
    if (V.ctl_h) __atomic_store_n(&V.ctl_h->shutdown, 1, __ATOMIC_RELEASE);
    int rc = SVM_OK;
    if (V.s_engine && cudaStreamSynchronize(V.s_engine) != cudaSuccess) rc = SVM_ERR_CUDA;
    for (auto &kv : V.jobs)
        if (kv.second->mem) cudaFreeAsync(kv.second->mem, V.s_side);
    if (V.s_side) cudaStreamSynchronize(V.s_side);
    for (void *p : {(void *)V.ctl_h, (void *)V.ring_h, (void *)V.slots_h, (void *)V.res_h, (void *)V.done_h,
                    (void *)V.info_h})
        if (p) cudaFreeHost(p);
    if (V.info_d) cudaFree(V.info_d);
    if (V.next_d) cudaFree(V.next_d);
    if (V.s_engine) cudaStreamDestroy(V.s_engine);
    if (V.s_side) cudaStreamDestroy(V.s_side);
    delete srv;
    return rc;
}

int svm_train_fixed_workspace(const svm_csr *X, const int8_t *y, const svm_params *params,
                              double *alpha_out, double *b_out, int64_t *iters_out)
{
    g_err.clear();
    try {
        return train_fixed_impl(X, y, params, alpha_out, b_out, iters_out);
    } catch (const Fail &f) {
        return f.code;
    } catch (...) {
        set_err("unexpected host exception");
        return SVM_ERR_CUDA;
    }
}

const char *svm_version(void) { return "svm_gb300 0.1 (sm_103a)"; }

}  // extern "C"
