// RBF contraction of query rows against the support vectors on CUDA cores:
//   out[q] = sum_k coef_k * exp(-gamma * (||z_q||^2 + ||x_k||^2 - 2 <z_q, x_k>))
//   (or, in the FP64 and mixed modes, K = a function of <z_q, x_k> for the
//   linear, polynomial and sigmoid kernels)
// This is the inner loop of gradient reconstruction (Algorithm 6, f of the
// shrunk samples from all alpha > 0) and of the decision function
// (Eq. classi). A CTA holds a tile of TQ query rows densified in shared
// memory (column-major, so one nonzero of a support vector gathers TQ
// consecutive words) and streams all support vectors; each thread owns a
// fixed subset of support vectors and the per-query partial sums are
// reduced in a fixed order, so results are deterministic.
#include <cuda_runtime.h>

#include "fp64_math.cuh"
#include "svm_internal.cuh"

namespace svmgb {
namespace {

constexpr int kCThreads = 256;
constexpr int kCWarps = kCThreads / 32;

template <int MODE, int TQ>
__global__ void __launch_bounds__(kCThreads) rbf_contract_kernel(RbfContract c)
{
    extern __shared__ __align__(16) unsigned char dsm[];
    __shared__ double red[kCWarps][TQ];
    __shared__ uint64_t expfx_s[MODE == MODE_FP64 ? kExpfxTabLen : 1];   // FP64: fixed-point exp
    __shared__ double zn[TQ];
    __shared__ int zlen[TQ];
    __shared__ int zrow[TQ];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int d = c.d;
    const int64_t qbase = (int64_t)blockIdx.x * TQ;
    const int nt = (int)min((int64_t)TQ, c.nq - qbase);

    // dense query tile, column-major: Zt[col * TQ + q]
    using Elem = typename std::conditional<MODE == MODE_FP64, double,
                 typename std::conditional<MODE == MODE_MIXED, float, unsigned>::type>::type;
    Elem *Zt = reinterpret_cast<Elem *>(dsm);
    const int tile_words = MODE == MODE_BINARY ? d : d * TQ;
    // FP64 with exact inner products: a tile entry holds (m, b) of the value
    // as two ints (xd_mant, xd_exp); an absent value is m = 0, b = tmin
    const bool xd = MODE == MODE_FP64 && c.xd.on;
    Elem zero = (Elem)0;
    if constexpr (MODE == MODE_FP64) {
        if (xd) zero = __hiloint2double(c.xd.tmin, 0);
    }
    for (int w = tid; w < tile_words; w += kCThreads) Zt[w] = zero;
    if constexpr (MODE == MODE_FP64) {
        for (int w = tid; w < kExpfxTabLen; w += kCThreads) expfx_s[w] = kExpfxTab[w];
    }
    if (tid < TQ) {
        int r = -1;
        if (tid < nt) r = c.q ? c.q[qbase + tid] : (int)(qbase + tid);
        zrow[tid] = r;
        if (r >= 0) {
            zlen[tid] = (int)(c.z_indptr[r + 1] - c.z_indptr[r]);
            zn[tid] = MODE == MODE_MIXED ? (double)c.z_normf[r] : (MODE == MODE_FP64 ? c.z_norm[r] : 0.0);
        } else {
            zlen[tid] = 0;
            zn[tid] = 0.0;
        }
    }
    __syncthreads();
    for (int q = 0; q < nt; ++q) {
        const int r = zrow[q];
        const int64_t p0 = c.z_indptr[r], p1 = c.z_indptr[r + 1];
        for (int64_t p = p0 + tid; p < p1; p += kCThreads) {
            const int col = c.z_indices[p];
            if constexpr (MODE == MODE_BINARY) atomicOr(&Zt[col], 1u << q);
            else if constexpr (MODE == MODE_FP64) {
                const float v = c.z_values[p];
                const uint32_t u = __float_as_uint(v);
                Zt[(size_t)col * TQ + q] = xd ? __hiloint2double(xd_exp(u, c.xd.tmin), xd_mant(u)) : widen_f32(v);
            }
            else Zt[(size_t)col * TQ + q] = (Elem)c.z_values[p];
        }
    }
    __syncthreads();

    double part[TQ];
#pragma unroll
    for (int q = 0; q < TQ; ++q) part[q] = 0.0;
    for (int64_t k = tid; k < c.nsv; k += kCThreads) {
        const int j = c.sv[k];
        const double coef = c.coef[k];
        const int64_t p0 = c.x_indptr[j], p1 = c.x_indptr[j + 1];
        if constexpr (MODE == MODE_BINARY) {
            int cnt[TQ];
#pragma unroll
            for (int q = 0; q < TQ; ++q) cnt[q] = 0;
            for (int64_t p = p0; p < p1; ++p) {
                const unsigned w = Zt[c.x_indices[p]];
#pragma unroll
                for (int q = 0; q < TQ; ++q) cnt[q] += (int)((w >> q) & 1u);
            }
            const int len = (int)(p1 - p0);
#pragma unroll
            for (int q = 0; q < TQ; ++q) {
                int dist = len + zlen[q] - 2 * cnt[q];
                dist = dist < 0 ? 0 : (dist >= c.ktab_len ? c.ktab_len - 1 : dist);
                part[q] = fma(coef, c.ktab[dist], part[q]);
            }
        } else if constexpr (MODE == MODE_FP64) {
            double acc[TQ];
            if (xd) {
                // exact inner products in integer arithmetic, rounded once
                XdAcc a[TQ];
#pragma unroll
                for (int q = 0; q < TQ; ++q) a[q] = xd_zero();
                const int2 *Z2 = reinterpret_cast<const int2 *>(Zt);
                for (int64_t p = p0; p < p1; ++p) {
                    const uint32_t u = __float_as_uint(c.x_values[p]);
                    const int32_t m = xd_mant(u);
                    const int e = xd_exp(u, c.xd.tmin) + c.xd.bias;
                    const int2 *zc = Z2 + (size_t)c.x_indices[p] * TQ;
#pragma unroll
                    for (int q = 0; q < TQ; ++q) {
                        const int2 t = zc[q];
                        xd_add(a[q], m, t.x, e + t.y);
                    }
                }
#pragma unroll
                for (int q = 0; q < TQ; ++q) acc[q] = xd_round(a[q], c.xd.unit);
            } else {
#pragma unroll
                for (int q = 0; q < TQ; ++q) acc[q] = 0.0;
                for (int64_t p = p0; p < p1; ++p) {
                    const double v = widen_f32(c.x_values[p]);
                    const double *zc = Zt + (size_t)c.x_indices[p] * TQ;
#pragma unroll
                    for (int q = 0; q < TQ; ++q) acc[q] = fma(v, zc[q], acc[q]);
                }
            }
            const double xn = c.x_norm[j];
            if (c.kernel == KERNEL_RBF) {
#pragma unroll
                for (int q = 0; q < TQ; ++q) {
                    double d2 = zn[q] + xn - 2.0 * acc[q];
                    part[q] = fma(coef, exp_neg_fx(c.gamma * (__double_as_longlong(d2) < 0 ? 0.0 : d2), expfx_s), part[q]);
                }
            } else {
#pragma unroll
                for (int q = 0; q < TQ; ++q)
                    part[q] = fma(coef, kernel_of_dot(c.kernel, c.gamma, c.coef0, c.degree, acc[q]), part[q]);
            }
        } else {
            float acc[TQ];
#pragma unroll
            for (int q = 0; q < TQ; ++q) acc[q] = 0.f;
            for (int64_t p = p0; p < p1; ++p) {
                const float v = c.x_values[p];
                const float *zc = Zt + (size_t)c.x_indices[p] * TQ;
#pragma unroll
                for (int q = 0; q < TQ; ++q) acc[q] = fmaf(v, zc[q], acc[q]);
            }
            const float xn = c.x_normf[j];
            const float g = (float)c.gamma;
            if (c.kernel == KERNEL_RBF) {
#pragma unroll
                for (int q = 0; q < TQ; ++q) {
                    float d2 = (float)zn[q] + xn - 2.0f * acc[q];
                    part[q] = fma(coef, (double)__expf(-g * fmaxf(d2, 0.f)), part[q]);
                }
            } else {
                const float c0 = (float)c.coef0;
#pragma unroll
                for (int q = 0; q < TQ; ++q)
                    part[q] = fma(coef, (double)kernel_of_dot(c.kernel, g, c0, c.degree, acc[q]), part[q]);
            }
        }
    }
    // fixed-order reduction: warp tree, then warps in order
#pragma unroll
    for (int q = 0; q < TQ; ++q) {
        double v = part[q];
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if (lane == 0) red[warp][q] = v;
    }
    __syncthreads();
    if (tid < nt) {
        double s = 0.0;
        for (int w = 0; w < kCWarps; ++w) s += red[w][tid];
        const int r = zrow[tid];
        double v = s + c.add_scalar;
        if (c.yq) v -= (double)c.yq[r];
        const int64_t o = c.out_by_row ? (int64_t)r : qbase + tid;
        if (c.accumulate) v = c.out[o] + v;
        c.out[o] = v;
    }
}

template <int MODE, int TQ>
cudaError_t launch_t(const RbfContract &c, cudaStream_t st)
{
    if (c.nq <= 0) return cudaSuccess;
    size_t smem = MODE == MODE_BINARY ? sizeof(unsigned) * (size_t)c.d
                                      : (MODE == MODE_FP64 ? sizeof(double) : sizeof(float)) * (size_t)c.d * TQ;
    auto fn = rbf_contract_kernel<MODE, TQ>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int64_t blocks = (c.nq + TQ - 1) / TQ;
    fn<<<(unsigned)blocks, kCThreads, smem, st>>>(c);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_rbf_contract(const RbfContract &c, cudaStream_t st)
{
    switch (c.mode) {
    case MODE_BINARY: return launch_t<MODE_BINARY, 16>(c, st);
    case MODE_FP64: return launch_t<MODE_FP64, 8>(c, st);
    case MODE_MIXED: return launch_t<MODE_MIXED, 8>(c, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace svmgb
