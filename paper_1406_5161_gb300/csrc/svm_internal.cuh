// Internal declarations of the GB300 SVM library (not part of the C ABI).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "svm_gb300.h"
#include "fp64_math.cuh"

namespace svmgb {

// Index sets of Eq. (setinfo), one byte per sample.
enum : uint8_t { ST_I0 = 0, ST_I1 = 1, ST_I2 = 2, ST_I3 = 3, ST_I4 = 4 };

__host__ __device__ __forceinline__ bool st_up(uint8_t s) { return s <= ST_I2; }
__host__ __device__ __forceinline__ bool st_low(uint8_t s) { return s == ST_I0 || s >= ST_I3; }
__host__ __device__ __forceinline__ uint8_t st_of(int8_t y, double a, double C)
{
    if (a > 0.0 && a < C) return ST_I0;
    if (a == 0.0) return y > 0 ? ST_I1 : ST_I4;
    return y > 0 ? ST_I3 : ST_I2;
}

// Row-pass arithmetic of the fused step.
enum { MODE_BINARY = 0, MODE_FP64 = 1, MODE_MIXED = 2, MODE_BITS4 = 3, MODE_BITS8 = 4 };

// Kernels (svm_kernel_kind). The RBF kernel is evaluated where its squared
// distance is formed; the others are functions of the inner product.
enum { KERNEL_RBF = 0, KERNEL_LINEAR = 1, KERNEL_POLY = 2, KERNEL_SIGMOID = 3 };

// linear <x,z>, polynomial (gamma <x,z> + coef0)^degree (power by repeated
// products), sigmoid tanh(gamma <x,z> + coef0); each FP64 operation rounded
// on its own, in this order
__device__ __forceinline__ double kernel_of_dot(int kind, double gamma, double coef0, int degree, double dot)
{
    if (kind == KERNEL_LINEAR) return dot;
    const double b = __dadd_rn(__dmul_rn(gamma, dot), coef0);
    if (kind == KERNEL_POLY) {
        double r = b;
        for (int k = 1; k < degree; ++k) r = __dmul_rn(r, b);
        return r;
    }
    return tanh(b);
}
__device__ __forceinline__ float kernel_of_dot(int kind, float gamma, float coef0, int degree, float dot)
{
    if (kind == KERNEL_LINEAR) return dot;
    const float b = __fadd_rn(__fmul_rn(gamma, dot), coef0);
    if (kind == KERNEL_POLY) {
        float r = b;
        for (int k = 1; k < degree; ++k) r = __fmul_rn(r, b);
        return r;
    }
    return tanhf(b);
}
// Binary rows held as bit masks of 4 or 8 words (d <= 128 or d <= 256): the
// squared distance of two binary rows is the popcount of their XOR.
__host__ __device__ constexpr bool mode_bits(int m) { return m == MODE_BITS4 || m == MODE_BITS8; }
__host__ __device__ constexpr int mode_words(int m) { return m == MODE_BITS8 ? 8 : 4; }

// Solver state carried between launches of the persistent step kernel.
struct SmoCtrl {
    double b_up, b_low;        // f at i_up / i_low over the active set
    double a_up, a_low;        // alpha of i_up / i_low
    int64_t iter;              // SMO steps done
    int64_t counter;           // shrink counter
    int64_t active;            // active-set size
    int64_t row_visits;        // sum of active-set sizes over the steps
    int32_t i_up, i_low;
    int32_t exit_reason;       // 0: gap <= thr, 1: iteration limit, 2: active set
                               // below SmoArgs::compact_below
    int32_t err;               // 0 ok, 1 timeout in a grid-wide wait
    int64_t shrink_events;
    // SM cycles spent by CTA 0 in each phase of a step (summed over steps,
    // recorded only when SmoArgs::phase_times is set):
    // 0 target rows, 1 pair step (FP64 part), 2 row pass + CTA reduction,
    // 3 publish, 4 grid exchange, 5 other, 6 pair step (K(up,low) part),
    // 7 second-order gain sweep and exchange
    int64_t phase_cycles[8];
    int64_t kc_hits, kc_misses;   // kernel-row cache lookups (CTA 0)
};

// Kernel arguments. Sample indices in the active lists are local to their
// segment (global index = seg_lo(segment) + local index).
struct SmoArgs {
    int64_t n;
    int32_t d;
    int32_t G;                 // CTAs = row segments
    const int64_t *indptr;
    const int32_t *indices;
    const float *values;       // FP64 mode
    const float *vmix;         // mixed mode: values rounded to BF16, held as FP32
    const uint32_t *ew;        // mixed mode, d < 2^16: each entry as one word, column in
                               // bits 0-15 and the BF16 value's bits in 16-31 (or NULL;
                               // required for rows held on chip)
    const uint64_t *ew64;      // FP64 mode with xd.on, d < 2^16: each entry as column
                               // (bits 0-15) and xd_word of its value (16-47), or NULL
    const int8_t *y;
    const double *norm;        // ||x_i||^2 (FP64 / binary: exact)
    const uint32_t *bits;      // bit-mask modes: row i = words [i * W, (i + 1) * W)
    const float *normf;        // mixed: ||x_i||^2 of the rounded values
    double *alpha;
    double *f;
    uint8_t *status;           // bits 0-2 index set, bit 7 label is +1
    int32_t *act;              // active lists, segment s at [lo(s), lo(s) + cnt(s))
    int32_t *seg_cnt;
    void *cand;                // smo_cand_slots(G) candidate slots of smo_cand_bytes() each
    unsigned *seq;             // [2][G], zeroed before each launch
    SmoCtrl *ctrl;
    int32_t *trace;            // [2 * trace_len]
    int64_t trace_len;
    const double *ktab;        // binary: exp(-gamma * k), k = 0 .. ktab_len - 1, followed by
                               // the correctly rounded 1 / (2 - 2 exp(-gamma * k)) (0 if <= 1e-12)
                               // and by 2 - 2 exp(-gamma * k)
    int32_t ktab_len;
    int32_t maxnnz;            // longest row
    int32_t resident;          // segments held in shared memory
    int32_t seg_rows_max;      // largest segment (rows)
    int64_t seg_nnz_max;       // largest segment (stored entries)
    double C, gamma, thr;
    int64_t iter_limit;
    int64_t h;                 // shrink counter reset value (0: no shrinking)
    int32_t select_only;       // start with a selection pass
    int32_t phase_times;       // record per-phase cycle counts (CTA 0)
    int64_t *cta_cycles;       // with phase_times: per-CTA cycles of work per launch (G)
    int64_t timeout_ns;
    // kernel-row cache (FP64 / mixed modes): kc_slots rows of kc_ld values
    // (double / float); each CTA stores and reads only its own segment's part
    // of a row; the directory lives in each CTA's shared memory (kc_direct:
    // slot = sample index, one valid bit per sample; else 4-way sets)
    void *kc;
    int64_t kc_ld;
    int32_t kc_slots;
    int32_t kc_direct;
    int32_t kernel, degree;    // kernel kind (KERNEL_*); polynomial degree
    double coef0;              // polynomial / sigmoid offset
    int32_t wss2;              // i_low by the second-order gain (its own kernel instantiation)
    // active-set re-layout: the launch ends (exit_reason 2) once fewer than
    // compact_below rows are active (0: never), so that the host can gather
    // the active rows into a smaller problem; gmap (NULL at the top level)
    // maps this problem's sample indices to the caller's for the trace and
    // the reported pair
    int64_t compact_below;
    const int32_t *gmap;
    // mixed mode, RBF: the rows as dense BF16 [n][d_pad] (d_pad a multiple of
    // 32, <= 256, zero padded) for the tensor-core row tiles; NULL = the CSR
    // row pass on the CUDA cores
    const __nv_bfloat16 *dmat;
    int32_t d_pad;
    // optional: (step, active rows) after each shrink event, 2 per event
    int64_t *atrace;
    int64_t atrace_len;
    // FP64 mode: inner products exact in 128-bit integers, rounded once
    // (xd.on), else FP64 sums in row order
    XdFormat xd;
};

// ---- batched and served solves: one job = one two-class problem
struct BatchJobDev {
    // the job's matrix (a batch shares one; a served job brings its own)
    const int64_t *indptr;
    const int32_t *indices;
    const float *values;       // FP64 mode
    const float *vmix;         // mixed mode (CSR)
    const __nv_bfloat16 *dmat; // mixed mode, dense rows: BF16 [rows][d]
    const double *norm;
    const float *normf;
    // the job's rows of that matrix, labels and state
    const int32_t *rows;
    const int8_t *y;
    double *alpha;
    double *f;
    uint8_t *status;
    int32_t nrows;
    int32_t d;                 // columns (dense: padded to a multiple of 8)
    int32_t dense;
    int32_t pad;
    double C, gamma, tau;
    int64_t max_iter;
    XdFormat xd;               // FP64 mode: exact inner products (xd.on)
};

struct BatchResultDev {
    double b, b_up, b_low, objective;
    int64_t iters;
    int32_t status;            // 0 converged, 1 iteration limit
    int32_t n_sv;
};

struct BatchArgs {
    int32_t d;                 // widest job (target buffers)
    int32_t njobs;             // static work-list: jobs[0 .. njobs)
    const BatchJobDev *jobs;   // job table (static list or server slots)
    BatchResultDev *results;   // per job / slot
    int *next_job;             // claim counter (zeroed before a static launch)
    int32_t ktab_len;          // binary mode: 2 * maxnnz + 1
    int32_t maxnnz;
    // dynamic work-list of a server (NULL for a batch): slots published by
    // the host in ring[head % ring_cap] for head < *ring_tail
    const int32_t *ring;
    const unsigned *ring_tail;
    int32_t ring_cap;
    int32_t pad;
    const int *shutdown;       // host sets to stop the engine
    int *done;                 // per slot: set to 1 when the result is written
    int64_t idle_ns;           // an engine cluster leaves after this long without work
};

size_t smo_batch_smem(int mode, int d, int ktab_len, int maxnnz);
int smo_batch_max_clusters(int mode, int lpr, int dense, size_t smem, int cs);
cudaError_t launch_smo_batch(int mode, int lpr, int dense, const BatchArgs &a, size_t smem, int cs,
                             int nclusters, cudaStream_t st);

// Dynamic shared-memory layout of the step kernel (byte offsets).
struct SmoLayout {
    size_t tgt, tcol, ktab, f, alpha, nrm, rowptr, act, st, col, val, bits, dist, kdir, frag, total;
};

__host__ __device__ inline size_t smo_align16(size_t x) { return (x + 15) & ~(size_t)15; }

__host__ __device__ inline SmoLayout smo_layout(int mode, int d, int ktab_len, int maxnnz,
                                                int resident, int rows, int64_t nnz, size_t kdir_bytes = 0)
{
    SmoLayout L;
    const bool bits = mode_bits(mode);
    size_t tgt_sz = bits ? 0 : (mode == 0 ? 2 : (mode == 1 ? 16 : 8));
    size_t o = 0;
    L.tgt = o;    o = smo_align16(o + 2 * (size_t)d * tgt_sz);
    L.tcol = o;   o = smo_align16(o + (bits ? 0 : 4 * (size_t)(maxnnz > 0 ? maxnnz : 1) * 4));
    L.ktab = o;   o = smo_align16(o + (mode == 0 || bits ? (size_t)ktab_len * 24 : 0));  // exp, 1/eta, eta tables
    if (!resident) rows = 0, nnz = 0;
    if (bits) nnz = 0;
    L.f = o;      o = smo_align16(o + (size_t)rows * 8);
    L.alpha = o;  o = smo_align16(o + (size_t)rows * 8);
    L.nrm = o;    o = smo_align16(o + (size_t)rows * (mode == 1 ? 8 : (mode == 2 ? 4 : 0)));
    L.rowptr = o; o = smo_align16(o + (size_t)(resident && !bits ? rows + 1 : 0) * 4);
    L.act = o;    o = smo_align16(o + (size_t)rows * 4);
    L.st = o;     o = smo_align16(o + (size_t)rows);
    // on-chip entries: FP64 a 16-bit column and an FP32 value; mixed one word
    // (column and BF16 value); binary the column
    L.col = o;    o = smo_align16(o + (size_t)nnz * (mode == 2 ? 0 : 2));
    L.val = o;    o = smo_align16(o + (size_t)nnz * (mode == 0 ? 0 : 4));
    L.bits = o;   o = smo_align16(o + (bits ? (size_t)rows * 4 * mode_words(mode) : 0));
    L.dist = o;   o = smo_align16(o + (bits ? (size_t)rows * 4 : 0));   // two 16-bit distances per row
    L.kdir = o;   o = smo_align16(o + kdir_bytes);                     // kernel-row cache directory
    // mixed mode: B fragments of the tensor-core row tiles (16 k-steps x 32 lanes x 8 B)
    L.frag = o;   o = smo_align16(o + (mode == 2 ? (size_t)16 * 32 * 8 : 0));
    L.total = o;
    return L;
}

__host__ __device__ __forceinline__ int64_t seg_lo(int64_t n, int G, int s)
{
    return (n * (int64_t)s) / G;
}

// ---------------------------------------------------------------- launchers
// (each returns a cudaError_t; kernels live in their own translation units)
// cs = CTAs per thread-block cluster (1, 8 or 16); G must be a multiple of cs
cudaError_t launch_smo_persistent(int mode, int lpr, const SmoArgs &a, size_t smem,
                                  cudaStream_t st, int cs);
// clusters of cs CTAs that can be resident at once (0 on error); resident:
// 0 streamed segments, 1 on-chip segments, 2 on-chip segments with the grid
// one cluster (the kernel that launch_smo_persistent picks when G == cs)
int smo_max_clusters(int mode, int lpr, int resident, size_t smem, int cs);
size_t smo_cand_bytes();   // bytes of one global candidate slot
// SFU exp2 instructions per second over the whole GPU (microbenchmark)
cudaError_t measure_sfu_ex2(double *ops_per_s, cudaStream_t st);
// one bounded wait on an mbarrier that nothing completes (failure-handling check)
cudaError_t launch_diag_wait(int64_t timeout_ns, const int *err, int *gave_up, cudaStream_t st);
// shared-memory bytes of a kernel-row cache directory
__host__ __device__ inline size_t smo_kdir_bytes(int64_t n, int slots, int direct)
{
    return direct ? (size_t)((n + 31) / 32) * 4 : (size_t)slots * 8;
}
// global exchange flags, kSeqStride words apart (a 128-byte line each): one
// per leader and epoch parity, then one per leader releasing its epochs to
// the FP64 kernel-row cache's cross-CTA reads; smo_seq_words(G) words
constexpr int kSeqStride = 32;
__host__ __device__ inline size_t smo_seq_words(int G) { return 3 * (size_t)G * kSeqStride; }
// global exchange slots of smo_cand_bytes() each for a launch of G CTAs: one
// per leader and epoch parity
__host__ __device__ inline size_t smo_cand_slots(int G) { return 2 * (size_t)G; }
size_t smo_static_smem(int mode);   // static shared memory of the step kernel of this mode
int smo_threads();

// Contraction of query rows against support vectors with the RBF epilogue:
//   out[q] = sum_k coef[k] * K(x_sv[k], z_q) + add_scalar - (yq ? yq[row] : 0)
// Gradient reconstruction (Algorithm 6) and the decision function
// (Eq. classi) are both this contraction.
struct RbfContract {
    // support vectors: rows sv[0..nsv) of X with coefficients alpha_k y_k
    const int64_t *x_indptr;
    const int32_t *x_indices;
    const float *x_values;     // FP64 mode: input values; mixed: BF16-rounded
    const double *x_norm;
    const float *x_normf;
    const int32_t *sv;
    const double *coef;
    int64_t nsv;
    // queries: rows q[0..nq) of Z, or rows 0..nq-1 when q == NULL
    const int64_t *z_indptr;
    const int32_t *z_indices;
    const float *z_values;
    const double *z_norm;
    const float *z_normf;
    const int32_t *q;
    int64_t nq;
    int32_t d;
    int32_t mode;              // MODE_BINARY / MODE_FP64 / MODE_MIXED
    double gamma;
    int32_t kernel, degree;    // kernel kind (KERNEL_*; binary and tensor-core paths: RBF)
    double coef0;
    const double *ktab;        // binary: exp(-gamma * k)
    int32_t ktab_len;
    int32_t out_by_row;        // 1: out[row id], 0: out[list position]
    double *out;
    const int8_t *yq;          // subtract yq[row] when non-NULL
    double add_scalar;
    int32_t accumulate;        // 1: add to out[] instead of writing (CUDA-core path only)
    XdFormat xd;               // FP64 mode: exact inner products (xd.on) for X and Z together
};
cudaError_t launch_rbf_contract(const RbfContract &c, cudaStream_t st);

// Tensor-core (tcgen05) version for MODE_MIXED inputs; d <= 256. `ws` holds
// tc_rbf_workspace_bytes(nq, nsv, d); *err_host is written asynchronously (1
// when a wait inside the kernel gave up) and is valid after a stream sync.
bool tc_rbf_supported(int d);
size_t tc_rbf_workspace_bytes(int64_t nq, int64_t nsv, int d);
cudaError_t launch_rbf_contract_tc(const RbfContract &c, void *ws, int *err_host, cudaStream_t st);

}  // namespace svmgb
