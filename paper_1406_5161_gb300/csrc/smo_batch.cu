// Batched SMO: many independent training jobs over one shared sample matrix
// in one persistent launch (one-vs-one subproblems, hyper-parameter grids).
//
// The grid is a set of thread-block clusters; each cluster takes the next
// job from a device work-list (an atomic counter), splits the job's rows
// over its CTAs and runs the job's SMO steps (Algorithm 1: Eqs. fup,
// bminmax, kktterm, alphaup) exactly as the single-job fused step does:
// target rows in shared memory, the FP64 pair step on warp 0 overlapped with
// the row sums of warps 1.., FP64 f updates, integer selection keys. The
// candidate exchange stays inside the cluster (distributed shared memory),
// so clusters never wait on one another and need no co-residency. When a
// job converges, the cluster reduces b (Section III-A) and the objective,
// writes the job's result and takes the next job.
//
// Rows of a job are ids into the shared matrix; the job's labels, alpha, f
// and index sets live in concatenated per-job arrays. Dense inputs in the
// mixed-precision mode are read from a BF16 row-major copy (2 bytes per
// value instead of 8 for index + value).
#include <cuda_bf16.h>

#include "smo_step.cuh"

namespace svmgb {
namespace smo {
namespace {

__device__ __forceinline__ unsigned ld_acquire_sys_u32(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_volatile_i32(const int *p)
{
    return *reinterpret_cast<const volatile int *>(p);
}
__device__ __forceinline__ void st_release_sys_i32(int *p, int v)
{
    asm volatile("st.release.sys.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

struct __align__(16) BatchFinish {
    double sum_a, sum_ayfy, sum_f0;
    long long n0, nsv;
    int pad[2];
};

// per warp: 16 k-steps x 32 lanes of packed BF16 target pairs (uint2)
constexpr size_t kFragBytes = (size_t)kWarps * 16 * 32 * sizeof(uint2);

struct BatchShared {
    Side wup[kWarps], wlow[kWarps];
    unsigned long long wkup[kWarps], wklow[kWarps];
    int wiup[kWarps], wilow[kWarps];
    CandFull ccand[kMaxCluster];   // cluster leader: its CTAs' candidates
    ResultArea res;
    BatchFinish fin[kMaxCluster];  // cluster leader: its CTAs' partial sums
    BatchFinish wfin[kWarps];
    double du, dl, au_new, al_new;
    unsigned char st_u, st_l;
    int job;
};

template <int MODE, int LPR>
__global__ void __launch_bounds__(kThreads, 1) smo_batch_kernel(BatchArgs B)
{
    using Tgt = typename RowMath<MODE>::Tgt;
    using Acc = typename RowMath<MODE>::Acc;
    extern __shared__ __align__(16) unsigned char dsm[];
    __shared__ BatchShared sh;
    // FP64: 2^(-j/256) in Q63 for the fixed-point exp
    __shared__ uint64_t expfx_s[MODE == MODE_FP64 ? kExpfxTabLen : 1];
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    const int csize = (int)cluster.num_blocks();
    const int crank = (int)cluster.block_rank();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int dmax = B.d;   // target buffers hold this many columns
    const int maxnnz = B.maxnnz > 0 ? B.maxnnz : 1;
    const SmoLayout L = smo_layout(MODE, dmax, B.ktab_len, maxnnz, 0, 0, 0);
    Tgt *tbuf = reinterpret_cast<Tgt *>(dsm + L.tgt);
    int *tcol = reinterpret_cast<int *>(dsm + L.tcol);
    double *ktab = reinterpret_cast<double *>(dsm + L.ktab);
    const double *rtab = ktab + B.ktab_len;
    if constexpr (MODE == MODE_FP64) {
        for (int c = tid; c < kExpfxTabLen; c += kThreads) expfx_s[c] = kExpfxTab[c];   // ordered by the cluster sync below
    }

    for (;;) {
        // ---- next job from the work-list, broadcast to the cluster
        if (crank == 0 && tid == 0) {
            int j = INT_MAX;
            if (!B.ring) {
                j = atomicAdd(B.next_job, 1);
                if (j >= B.njobs) j = INT_MAX;
            } else {
                // server: wait (bounded by the idle limit) for a published slot
                const uint64_t t0 = global_ns();
                for (;;) {
                    const unsigned tail = ld_acquire_sys_u32(B.ring_tail);
                    const unsigned head = (unsigned)atomicAdd(B.next_job, 0);
                    if (head < tail) {
                        if ((unsigned)atomicCAS(B.next_job, (int)head, (int)(head + 1)) == head) {
                            j = ld_volatile_i32(B.ring + (head % (unsigned)B.ring_cap));
                            break;
                        }
                        continue;
                    }
                    if (ld_volatile_i32(B.shutdown)) break;
                    if (global_ns() - t0 > (uint64_t)B.idle_ns) break;
                    __nanosleep(2000);
                }
            }
            for (int r = 0; r < csize; ++r) *cluster.map_shared_rank(&sh.job, r) = j;
        }
        cluster.sync();
        const int job = sh.job;
        if (job == INT_MAX) break;
        const BatchJobDev J = B.jobs[job];
        // the job's matrix (shared by all jobs of a batch, own per served job)
        const int d = J.d;
        const bool dense = J.dense != 0;
        const int64_t *indptr = J.indptr;
        const int32_t *indices = J.indices;
        const float *values = J.values;
        const float *vmix = J.vmix;
        const __nv_bfloat16 *dmat = J.dmat;
        const double *norm = J.norm;
        const float *normf = J.normf;
        const int m = J.nrows;
        const int8_t *yj = J.y;
        double *aj = J.alpha;
        double *fj = J.f;
        uint8_t *sj = J.status;
        const int lo = (int)((int64_t)m * crank / csize);
        const int hi = (int)((int64_t)m * (crank + 1) / csize);
        const double C = J.C, gamma = J.gamma;
        const float gammaf = (float)gamma;
        const double snap = 1e-12 * C, c_snap = C - snap;
        const double thr = 2.0 * J.tau;
        const int32_t *rows = J.rows;

        // FP64 with exact inner products (J.xd.on): target entries hold (m, b)
        // pairs as in the single-solve kernel; an absent value m = 0, b = tmin
        const bool xd = MODE == MODE_FP64 && J.xd.on;
        const int xd_tmin = J.xd.tmin, xd_bias = J.xd.bias, xd_unit = J.xd.unit;
        Tgt tclear;
        tgt_clear<MODE>(tclear);
        if constexpr (MODE == MODE_FP64) {
            if (xd) tclear = make_double2(__hiloint2double(xd_tmin, 0), __hiloint2double(xd_tmin, 0));
        }
        // ---- job set-up: tables, empty target buffers, alpha = 0, f = -y
        for (int c = tid; c < 2 * dmax; c += kThreads) tbuf[c] = tclear;
        if constexpr (MODE == MODE_BINARY) {
            for (int k = tid; k < B.ktab_len; k += kThreads) {
                const double kv = exp(-gamma * (double)k);
                const double eta = 2.0 - 2.0 * kv;
                ktab[k] = kv;
                ktab[B.ktab_len + k] = eta > 1e-12 ? 1.0 / eta : 0.0;
            }
        }
        for (int r = lo + tid; r < hi; r += kThreads) {
            const int8_t yr = yj[r];
            aj[r] = 0.0;
            fj[r] = -(double)yr;
            sj[r] = (uint8_t)(st_of(yr, 0.0, 1.0) | (yr > 0 ? 0x80 : 0));
        }
        __syncthreads();

        Side up, low;
        side_empty(up, true);
        side_empty(low, false);
        bool first = true;
        int64_t iter = 0;
        int prev_valid = 0, prev_len_u = 0, prev_len_l = 0;
        int64_t prev_pu = 0, prev_pl = 0;
        int status_code = 0;
        for (;;) {
            const int buf = (int)(iter & 1);
            Tgt *T = tbuf + (size_t)buf * dmax;
            int *tcu = tcol + (size_t)(buf * 2 + 0) * maxnnz;
            int *tcl = tcol + (size_t)(buf * 2 + 1) * maxnnz;
            if (!first) {
                if (!dless(thr, low.f - up.f)) { status_code = 0; break; }
                if (iter >= J.max_iter) { status_code = 1; break; }
                // ---- 1. targets into the shared-memory buffer
                if (dense) {
                    if constexpr (MODE == MODE_MIXED) {
                        const __nv_bfloat16 *ru = dmat + (size_t)up.p0 * d;
                        const __nv_bfloat16 *rl = dmat + (size_t)low.p0 * d;
                        for (int c = tid; c < d; c += kThreads) {
                            T[c].x = __bfloat162float(ru[c]);
                            T[c].y = __bfloat162float(rl[c]);
                        }
                    }
                } else {
                    // x_up by the first half of the threads, x_low by the
                    // second: both rows' loads in flight together
                    constexpr int kHalf = kThreads / 2;
                    if (tid < kHalf) {
                        for (int k = tid; k < up.len; k += kHalf) {
                            const int c = indices[up.p0 + k];
                            tcu[k] = c;
                            if constexpr (MODE == MODE_BINARY) reinterpret_cast<unsigned char *>(T + c)[0] = 1;
                            else if constexpr (MODE == MODE_FP64) xd_put<0>(T[c], values[up.p0 + k], xd, xd_tmin, 0);
                            else T[c].x = vmix[up.p0 + k];
                        }
                    } else {
                        for (int k = tid - kHalf; k < low.len; k += kHalf) {
                            const int c = indices[low.p0 + k];
                            tcl[k] = c;
                            if constexpr (MODE == MODE_BINARY) reinterpret_cast<unsigned char *>(T + c)[1] = 1;
                            else if constexpr (MODE == MODE_FP64) xd_put<1>(T[c], values[low.p0 + k], xd, xd_tmin, 0);
                            else T[c].y = vmix[low.p0 + k];
                        }
                    }
                }
                __syncthreads();
            }
            unsigned long long bku = kNoKey, bkl = kNoKey;
            int biu = INT_MAX, bil = INT_MAX, bru = 0, brl = 0;
            if (warp == 0) {
                // ---- 2. pair step (Eq. alphaup with rho = -eta, Platt clip)
                if (!first) {
                    Acc s = 0;
                    if (dense) {
                        if constexpr (MODE == MODE_MIXED)
                            for (int c = lane; c < d; c += 32) s = fmaf(T[c].y, T[c].x, s);
                    } else if (xd) {
                        if constexpr (MODE == MODE_FP64) {
                            const int4 *T4 = reinterpret_cast<const int4 *>(T);
                            XdAcc a = xd_zero();
                            for (int k = lane; k < low.len; k += 32) {
                                const int4 t = T4[tcl[k]];
                                xd_add(a, t.z, t.x, t.w + t.y + xd_bias);
                            }
                            xd_lane_sum<32>(a);
                            s = xd_round(a, xd_unit);
                        }
                    } else {
                        for (int k = lane; k < low.len; k += 32) {
                            const Tgt t = T[tcl[k]];
                            if constexpr (MODE == MODE_BINARY) s += (int)(t & 1);
                            else if constexpr (MODE == MODE_FP64) s = fma(t.y, t.x, s);
                            else s = fmaf(t.y, t.x, s);
                        }
                    }
                    if (!xd) {
#pragma unroll
                        for (int o = 16; o >= 1; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
                    }
                    if (lane == 0) {
                        double kul, rinv = 0.0;
                        if constexpr (MODE == MODE_BINARY) {
                            int dist = up.len + low.len - 2 * s;
                            dist = dist < 0 ? 0 : dist;
                            kul = ktab[dist];
                            rinv = rtab[dist];
                        } else if constexpr (MODE == MODE_FP64) {
                            double d2 = up.nrm + low.nrm - 2.0 * s;
                            kul = exp_neg_fx(gamma * dpos(d2), expfx_s);
                        } else {
                            float d2 = (float)up.nrm + (float)low.nrm - 2.0f * s;
                            kul = (double)__expf(-gammaf * fmaxf(d2, 0.f));
                        }
                        const bool yu_neg = up.y < 0, yl_neg = low.y < 0;
                        const double au = up.a, al = low.a;
                        const double eta = 2.0 - 2.0 * kul;
                        const bool opposite = yu_neg != yl_neg;
                        double Lo, Hi;
                        if (opposite) {
                            const double x = al - au;
                            Lo = dless(x, 0.0) ? 0.0 : x;
                            const double h = C + al - au;
                            Hi = dless(h, C) ? h : C;
                        } else {
                            const double x = al + au - C;
                            Lo = dless(x, 0.0) ? 0.0 : x;
                            const double h = al + au;
                            Hi = dless(h, C) ? h : C;
                        }
                        const double slope = neg_if(up.f - low.f, yl_neg);
                        double aln;
                        if (dless(1e-12, eta)) {
                            double q;
                            if constexpr (MODE == MODE_BINARY) {
                                const double q0 = slope * rinv;
                                const double rr = fma(-eta, q0, slope);
                                q = fma(rr, rinv, q0);
                            } else {
                                q = slope / eta;
                            }
                            const double t = al + q;
                            aln = dless(t, Lo) ? Lo : (dless(Hi, t) ? Hi : t);
                        } else {
                            aln = dless(0.0, slope) ? Hi : Lo;
                        }
                        double aun = au + neg_if(al - aln, opposite);
                        if (dless(aln, snap)) aln = 0.0;
                        if (dless(c_snap, aln)) aln = C;
                        if (dless(aun, snap)) aun = 0.0;
                        if (dless(c_snap, aun)) aun = C;
                        sh.du = neg_if(aun - au, yu_neg);
                        sh.dl = neg_if(aln - al, yl_neg);
                        sh.au_new = aun;
                        sh.al_new = aln;
                        sh.st_u = status_of(!yu_neg, aun, C);
                        sh.st_l = status_of(!yl_neg, aln, C);
                    }
                    __syncwarp();
                    step_bar_arrive(kThreads);
                }
            } else {
                // ---- 3. row pass over this CTA's rows of the job
                constexpr int kRowWarps = kWarps - 1;
                double du = 0.0, dl = 0.0, au_new = 0.0, al_new = 0.0;
                unsigned char st_u = 0, st_l = 0;
                bool have_step = first;
                auto wait_step = [&]() {
                    if (!have_step) {
                        step_bar_sync(kThreads);
                        du = sh.du; dl = sh.dl;
                        st_u = sh.st_u; st_l = sh.st_l;
                        au_new = sh.au_new; al_new = sh.al_new;
                        have_step = true;
                    }
                };
                // kernel values, FP64 update of Eq. (fup), selection keys of one row
                auto finish_row = [&](int r, int g, int len, Acc su, Acc sl, double fi, uint8_t sb) {
                    if (!first) {
                        double ku, kl;
                        if constexpr (MODE == MODE_BINARY) {
                            int du2 = up.len + len - 2 * su, dl2 = low.len + len - 2 * sl;
                            ku = ktab[du2 < 0 ? 0 : du2];
                            kl = ktab[dl2 < 0 ? 0 : dl2];
                        } else if constexpr (MODE == MODE_FP64) {
                            const double nrm_i = norm[g];
                            double d2u = up.nrm + nrm_i - 2.0 * su;
                            double d2l = low.nrm + nrm_i - 2.0 * sl;
                            ku = exp_neg_fx(gamma * dpos(d2u), expfx_s);
                            kl = exp_neg_fx(gamma * dpos(d2l), expfx_s);
                        } else {
                            const float nf = normf[g];
                            float d2u = (float)up.nrm + nf - 2.0f * su;
                            float d2l = (float)low.nrm + nf - 2.0f * sl;
                            // widened exactly by integer operations (a conversion
                            // instruction would take a slot of the FP64 pipe)
                            ku = widen_f32(__expf(-gammaf * fmaxf(d2u, 0.f)));
                            kl = widen_f32(__expf(-gammaf * fmaxf(d2l, 0.f)));
                        }
                        fi = fma(dl, kl, fma(du, ku, fi));
                        fj[r] = fi;
                        if (r == up.i) {
                            sb = st_u;
                            sj[r] = sb;
                            aj[r] = au_new;
                        } else if (r == low.i) {
                            sb = st_l;
                            sj[r] = sb;
                            aj[r] = al_new;
                        }
                    }
                    const uint8_t set = set_bits(sb);
                    const unsigned long long kup = key_up(fi), klo = key_low(fi);
                    if (st_up(set) && ki_less(kup, r, bku, biu)) { bku = kup; biu = r; bru = r; }
                    if (st_low(set) && ki_less(klo, r, bkl, bil)) { bkl = klo; bil = r; brl = r; }
                };
                bool blocked = false;
                if constexpr (LPR == 32) blocked = dense && d <= 256;
                bool tiles = false;   // dense BF16 rows on the tensor cores
                if constexpr (LPR == 16 && MODE == MODE_MIXED) tiles = dense && (d & 31) == 0 && d <= 256;
                if (tiles) {
                    if constexpr (LPR == 16 && MODE == MODE_MIXED) {
                        // Tiles of 16 rows x the two target rows on the
                        // tensor cores (mma m16n8k16, BF16 inputs, FP32
                        // accumulation; columns 2..7 of B are zero). Inside
                        // each 32-column block the K order is permuted so
                        // that a thread reads 8 consecutive values of a row
                        // with one 16-byte load: in k-step h of the block,
                        // logical k = 2t + i maps to column 8t + 4h + i and
                        // k = 2t + 8 + i to 8t + 4h + 2 + i; the targets use
                        // the same map, so the dot products are unchanged.
                        const int g = lane >> 2, t = lane & 3;
                        const int nblk = d >> 5;
                        // this warp's target fragments: [k-step][lane], k-step = 2 * block + h
                        uint2 *frag = reinterpret_cast<uint2 *>(dsm + L.total) + (size_t)warp * 16 * 32;
#pragma unroll
                        for (int b = 0; b < 8; ++b) {
#pragma unroll
                            for (int h = 0; h < 2; ++h) {
                                uint32_t r0 = 0, r1 = 0;
                                if (!first && g < 2 && b < nblk) {
                                    const int c = 32 * b + 8 * t + 4 * h;
                                    float e[4];
#pragma unroll
                                    for (int x = 0; x < 4; ++x) e[x] = g == 0 ? T[c + x].x : T[c + x].y;
                                    const __nv_bfloat162 p0 = __floats2bfloat162_rn(e[0], e[1]);
                                    const __nv_bfloat162 p1 = __floats2bfloat162_rn(e[2], e[3]);
                                    r0 = *reinterpret_cast<const uint32_t *>(&p0);
                                    r1 = *reinterpret_cast<const uint32_t *>(&p1);
                                }
                                frag[(2 * b + h) * 32 + lane] = make_uint2(r0, r1);
                            }
                        }
                        __syncwarp();
                        for (int base = lo + (warp - 1) * 16;; base += kRowWarps * 16) {
                            const bool round0 = base == lo + (warp - 1) * 16;
                            if (!round0 && base >= hi) break;
                            const int ra = base + g, rb = base + g + 8;
                            float acc[4] = {0.f, 0.f, 0.f, 0.f};
                            if (!first) {
                                const __nv_bfloat16 *pa = ra < hi ? dmat + (size_t)rows[ra] * d + 8 * t : nullptr;
                                const __nv_bfloat16 *pb = rb < hi ? dmat + (size_t)rows[rb] * d + 8 * t : nullptr;
                                // all blocks' loads in flight before their MMAs
#pragma unroll
                                for (int b0 = 0; b0 < 8; b0 += 8) {
                                    uint4 uu[8], vv[8];
#pragma unroll
                                    for (int q = 0; q < 8; ++q) {
                                        const int b = b0 + q;
                                        uu[q] = (pa && b < nblk) ? __ldg(reinterpret_cast<const uint4 *>(pa + 32 * b)) : make_uint4(0, 0, 0, 0);
                                        vv[q] = (pb && b < nblk) ? __ldg(reinterpret_cast<const uint4 *>(pb + 32 * b)) : make_uint4(0, 0, 0, 0);
                                    }
#pragma unroll
                                    for (int q = 0; q < 8; ++q) {
                                    const int b = b0 + q;
                                    if (b < nblk) {
                                        const uint4 u = uu[q], v = vv[q];
                                        const uint2 f0 = frag[(2 * b) * 32 + lane], f1 = frag[(2 * b + 1) * 32 + lane];
                                        asm volatile(
                                            "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
                                            "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                                            : "+f"(acc[0]), "+f"(acc[1]), "+f"(acc[2]), "+f"(acc[3])
                                            : "r"(u.x), "r"(v.x), "r"(u.y), "r"(v.y), "r"(f0.x), "r"(f0.y));
                                        asm volatile(
                                            "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
                                            "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                                            : "+f"(acc[0]), "+f"(acc[1]), "+f"(acc[2]), "+f"(acc[3])
                                            : "r"(u.z), "r"(v.z), "r"(u.w), "r"(v.w), "r"(f1.x), "r"(f1.y));
                                    }
                                    }
                                }
                            }
                            // lanes with t == 0 hold the two sums of rows ra and rb
                            const bool lead = t == 0;
                            double fa = 0.0, fb = 0.0;
                            uint8_t sa = 0, sbb = 0;
                            int ga = 0, gb = 0;
                            if (lead && ra < hi) { ga = rows[ra]; fa = fj[ra]; sa = sj[ra]; }
                            if (lead && rb < hi) { gb = rows[rb]; fb = fj[rb]; sbb = sj[rb]; }
                            wait_step();
                            if (lead && ra < hi) finish_row(ra, ga, d, acc[0], acc[1], fa, sa);
                            if (lead && rb < hi) finish_row(rb, gb, d, acc[2], acc[3], fb, sbb);
                        }
                    }
                } else if (blocked) {
                    if constexpr (LPR == 32 && MODE == MODE_MIXED) {
                        // 8 rows per warp at a time; lane l covers columns
                        // [8l, 8l+8) of all 8 rows with its target columns in
                        // registers; a butterfly transpose-reduction leaves
                        // each group of 4 lanes with one row's two sums
                        const int c8 = lane * 8;
                        const bool has_cols = c8 < d;
                        float tu[8], tl[8];
#pragma unroll
                        for (int e = 0; e < 8; ++e) {
                            tu[e] = 0.f;
                            tl[e] = 0.f;
                        }
                        if (!first && has_cols) {
#pragma unroll
                            for (int e = 0; e < 8; ++e) {
                                const float2 t = T[c8 + e];
                                tu[e] = t.x;
                                tl[e] = t.y;
                            }
                        }
                        const bool h16 = (lane & 16) != 0, h8 = (lane & 8) != 0, h4 = (lane & 4) != 0;
                        const int ri = (h16 ? 4 : 0) + (h8 ? 2 : 0) + (h4 ? 1 : 0);
                        for (int base = lo + (warp - 1) * 8;; base += kRowWarps * 8) {
                            const bool round0 = base == lo + (warp - 1) * 8;
                            if (!round0 && base >= hi) break;
                            float pu[8], pl[8];
#pragma unroll
                            for (int j = 0; j < 8; ++j) {
                                pu[j] = 0.f;
                                pl[j] = 0.f;
                                const int r = base + j;
                                if (!first && r < hi && has_cols) {
                                    const int g = rows[r];
                                    const uint4 raw = *reinterpret_cast<const uint4 *>(dmat + (size_t)g * d + c8);
                                    const __nv_bfloat162 *h2 = reinterpret_cast<const __nv_bfloat162 *>(&raw);
#pragma unroll
                                    for (int e = 0; e < 4; ++e) {
                                        const float2 v = __bfloat1622float2(h2[e]);
                                        pu[j] = fmaf(v.x, tu[2 * e], pu[j]);
                                        pl[j] = fmaf(v.x, tl[2 * e], pl[j]);
                                        pu[j] = fmaf(v.y, tu[2 * e + 1], pu[j]);
                                        pl[j] = fmaf(v.y, tl[2 * e + 1], pl[j]);
                                    }
                                }
                            }
                            float au[4], al[4];
#pragma unroll
                            for (int k = 0; k < 4; ++k) {
                                au[k] = (h16 ? pu[k + 4] : pu[k]) + __shfl_xor_sync(0xffffffffu, h16 ? pu[k] : pu[k + 4], 16);
                                al[k] = (h16 ? pl[k + 4] : pl[k]) + __shfl_xor_sync(0xffffffffu, h16 ? pl[k] : pl[k + 4], 16);
                            }
                            float bu2[2], bl2[2];
#pragma unroll
                            for (int k = 0; k < 2; ++k) {
                                bu2[k] = (h8 ? au[k + 2] : au[k]) + __shfl_xor_sync(0xffffffffu, h8 ? au[k] : au[k + 2], 8);
                                bl2[k] = (h8 ? al[k + 2] : al[k]) + __shfl_xor_sync(0xffffffffu, h8 ? al[k] : al[k + 2], 8);
                            }
                            float su = (h4 ? bu2[1] : bu2[0]) + __shfl_xor_sync(0xffffffffu, h4 ? bu2[0] : bu2[1], 4);
                            float sl = (h4 ? bl2[1] : bl2[0]) + __shfl_xor_sync(0xffffffffu, h4 ? bl2[0] : bl2[1], 4);
                            su += __shfl_xor_sync(0xffffffffu, su, 2);
                            sl += __shfl_xor_sync(0xffffffffu, sl, 2);
                            su += __shfl_xor_sync(0xffffffffu, su, 1);
                            sl += __shfl_xor_sync(0xffffffffu, sl, 1);
                            const int r = base + ri;
                            double fi = 0.0;
                            uint8_t sb = 0;
                            int g = 0;
                            const bool lead = (lane & 3) == 0 && r < hi;
                            if (lead) {
                                g = rows[r];
                                fi = fj[r];
                                sb = sj[r];
                            }
                            wait_step();
                            if (lead) finish_row(r, g, d, su, sl, fi, sb);
                        }
                    }
                } else {
                    constexpr int RPW = 32 / LPR;
                    const int gl = lane & (LPR - 1);
                    const int gw = lane / LPR;
                    for (int kb = lo + (warp - 1) * RPW;; kb += kRowWarps * RPW) {
                        const bool round0 = kb == lo + (warp - 1) * RPW;
                        if (!round0 && kb >= hi) break;
                        const int r = kb + gw;
                        const bool valid = r < hi;
                        int g = 0;
                        int64_t p0 = 0, p1 = 0;
                        double fi = 0.0;
                        uint8_t sb = 0;
                        if (valid) {
                            g = rows[r];
                            if (!dense) {
                                p0 = indptr[g];
                                p1 = indptr[g + 1];
                            }
                            if (gl == 0) {
                                fi = fj[r];
                                sb = sj[r];
                            }
                        }
                        Acc su = 0, sl = 0;
                        XdAcc au = xd_zero(), al = xd_zero();   // FP64, exact inner products
                        if (!first && valid) {
                            if (dense) {
                                if constexpr (MODE == MODE_MIXED) {
                                const __nv_bfloat16 *xr = dmat + (size_t)g * d;
                                for (int c = gl * 8; c < d; c += LPR * 8) {
                                    const uint4 raw = *reinterpret_cast<const uint4 *>(xr + c);
                                    const __nv_bfloat162 *h2 = reinterpret_cast<const __nv_bfloat162 *>(&raw);
#pragma unroll
                                    for (int e = 0; e < 4; ++e) {
                                        const float2 v = __bfloat1622float2(h2[e]);
                                        const float2 t0 = T[c + 2 * e], t1 = T[c + 2 * e + 1];
                                        su = fmaf(v.x, t0.x, su);
                                        sl = fmaf(v.x, t0.y, sl);
                                        su = fmaf(v.y, t1.x, su);
                                        sl = fmaf(v.y, t1.y, sl);
                                    }
                                }
                                }
                            } else if (xd) {
                                if constexpr (MODE == MODE_FP64) {
                                    const int4 *T4 = reinterpret_cast<const int4 *>(T);
                                    for (int64_t p = p0 + gl; p < p1; p += LPR) {
                                        const uint32_t u = __float_as_uint(values[p]);
                                        const int32_t mx = xd_mant(u);
                                        const int e = xd_exp(u, xd_tmin) + xd_bias;
                                        const int4 t = T4[indices[p]];
                                        xd_add(au, mx, t.x, e + t.y);
                                        xd_add(al, mx, t.z, e + t.w);
                                    }
                                }
                            } else {
                                for (int64_t p = p0 + gl; p < p1; p += LPR) {
                                    const int c = indices[p];
                                    if constexpr (MODE == MODE_BINARY) {
                                        const unsigned short t = T[c];
                                        su += (int)(t & 0xff);
                                        sl += (int)(t >> 8);
                                    } else if constexpr (MODE == MODE_FP64) {
                                        const double v = (double)values[p];
                                        const double2 t = T[c];
                                        su = fma(v, t.x, su);
                                        sl = fma(v, t.y, sl);
                                    } else {
                                        const float v = vmix[p];
                                        const float2 t = T[c];
                                        su = fmaf(v, t.x, su);
                                        sl = fmaf(v, t.y, sl);
                                    }
                                }
                            }
                        }
                        if (!first && xd) {
                            if constexpr (MODE == MODE_FP64) {
                                xd_lane_sum<LPR>(au);
                                xd_lane_sum<LPR>(al);
                                su = xd_round(au, xd_unit);
                                sl = xd_round(al, xd_unit);
                            }
                        } else if (!first) {
#pragma unroll
                            for (int o = LPR / 2; o >= 1; o >>= 1) {
                                su += __shfl_xor_sync(0xffffffffu, su, o);
                                sl += __shfl_xor_sync(0xffffffffu, sl, o);
                            }
                        }
                        wait_step();
                        if (valid && gl == 0) finish_row(r, g, (int)(p1 - p0), su, sl, fi, sb);
                    }
                }
            }
            // payload of a job row (job-local index r)
            auto make_side = [&](int r) {
                Side sd;
                const int g = rows[r];
                const uint8_t sb = sj[r];
                sd.f = fj[r];
                sd.a = aj[r];
                if constexpr (MODE == MODE_FP64) sd.nrm = norm[g];
                else if constexpr (MODE == MODE_MIXED) sd.nrm = (double)normf[g];
                else sd.nrm = 0.0;
                if (dense) {
                    sd.p0 = g;
                    sd.len = d;
                } else {
                    sd.p0 = indptr[g];
                    sd.len = (int)(indptr[g + 1] - sd.p0);
                }
                sd.i = r;
                sd.y = y_of(sb);
                sd.owner = 0;
                return sd;
            };
            {
                unsigned long long k1 = bku, k2 = bkl;
                int i1 = biu, i2 = bil;
                warp_min_ki(k1, i1);
                warp_min_ki(k2, i2);
                if (lane == 0) {
                    sh.wkup[warp] = k1; sh.wiup[warp] = i1;
                    sh.wklow[warp] = k2; sh.wilow[warp] = i2;
                }
                if (i1 != INT_MAX && biu == i1) sh.wup[warp] = make_side(bru);
                if (i2 != INT_MAX && bil == i2) sh.wlow[warp] = make_side(brl);
            }
            __syncthreads();
            // ---- 4. candidate exchange inside the cluster
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
                if (lane == 0) {
                    CandFull cf;
                    if (mu) cf.up = sh.wup[__ffs(mu) - 1]; else side_empty(cf.up, true);
                    if (ml) cf.low = sh.wlow[__ffs(ml) - 1]; else side_empty(cf.low, false);
                    cf.count = hi - lo;
                    cf.pad[0] = cf.pad[1] = cf.pad[2] = 0;
                    *(cluster.map_shared_rank(sh.ccand, 0) + crank) = cf;
                }
            }
            if (prev_valid && warp >= 8) {
                Tgt *P = tbuf + (size_t)(1 - buf) * dmax;
                if (dense) {
                    (void)prev_pu;
                    (void)prev_pl;
                } else {
                    const int *pcu = tcol + (size_t)((1 - buf) * 2 + 0) * maxnnz;
                    const int *pcl = tcol + (size_t)((1 - buf) * 2 + 1) * maxnnz;
                    for (int k = tid - 256; k < prev_len_u; k += kThreads - 256) P[pcu[k]] = tclear;
                    for (int k = tid - 256; k < prev_len_l; k += kThreads - 256) P[pcl[k]] = tclear;
                }
            }
            cluster.sync();
            if (crank == 0 && warp == 0) {
                CandFull c;
                if (lane < csize) c = sh.ccand[lane];
                else { side_empty(c.up, true); side_empty(c.low, false); c.count = 0; }
                unsigned long long k1 = c.up.i == INT_MAX ? kNoKey : key_up(c.up.f);
                unsigned long long k2 = c.low.i == INT_MAX ? kNoKey : key_low(c.low.f);
                int i1 = c.up.i, i2 = c.low.i;
                const unsigned long long k1s = k1, k2s = k2;
                const int i1s = i1, i2s = i2;
                warp_min_ki(k1, i1);
                warp_min_ki(k2, i2);
                const unsigned mu = __ballot_sync(0xffffffffu, i1 != INT_MAX && k1s == k1 && i1s == i1);
                const unsigned ml = __ballot_sync(0xffffffffu, i2 != INT_MAX && k2s == k2 && i2s == i2);
                if (lane < csize) {
                    ResultArea res;
                    if (mu) res.up = sh.ccand[__ffs(mu) - 1].up; else side_empty(res.up, true);
                    if (ml) res.low = sh.ccand[__ffs(ml) - 1].low; else side_empty(res.low, false);
                    res.total = m;
                    res.flag = 0;
                    res.gap_open = 1;   // the batch kernel tests the gap itself
                    *cluster.map_shared_rank(&sh.res, lane) = res;
                }
            }
            cluster.sync();
            prev_valid = first ? 0 : 1;
            prev_len_u = up.len;
            prev_len_l = low.len;
            prev_pu = up.p0;
            prev_pl = low.p0;
            up = sh.res.up;
            low = sh.res.low;
            if (!first) ++iter;
            first = false;
        }

        // ---- job results: b (Section III-A) and the objective from partial sums
        {
            BatchFinish pf = {0, 0, 0, 0, 0, {0, 0}};
            for (int r = lo + tid; r < hi; r += kThreads) {
                const double a = aj[r];
                const uint8_t sb = sj[r];
                const double yi = (sb & 0x80) ? 1.0 : -1.0;
                const double fi = fj[r];
                pf.sum_a += a;
                pf.sum_ayfy += a * yi * (fi + yi);
                if ((sb & 7) == ST_I0) { pf.sum_f0 += fi; pf.n0 += 1; }
                if (a > 0.0) pf.nsv += 1;
            }
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) {
                pf.sum_a += __shfl_xor_sync(0xffffffffu, pf.sum_a, o);
                pf.sum_ayfy += __shfl_xor_sync(0xffffffffu, pf.sum_ayfy, o);
                pf.sum_f0 += __shfl_xor_sync(0xffffffffu, pf.sum_f0, o);
                pf.n0 += __shfl_xor_sync(0xffffffffu, pf.n0, o);
                pf.nsv += __shfl_xor_sync(0xffffffffu, pf.nsv, o);
            }
            if (lane == 0) sh.wfin[warp] = pf;
            __syncthreads();
            if (tid == 0) {
                BatchFinish t = sh.wfin[0];
                for (int w = 1; w < kWarps; ++w) {
                    t.sum_a += sh.wfin[w].sum_a;
                    t.sum_ayfy += sh.wfin[w].sum_ayfy;
                    t.sum_f0 += sh.wfin[w].sum_f0;
                    t.n0 += sh.wfin[w].n0;
                    t.nsv += sh.wfin[w].nsv;
                }
                *(cluster.map_shared_rank(sh.fin, 0) + crank) = t;
            }
            cluster.sync();
            if (crank == 0 && tid == 0) {
                BatchFinish t = sh.fin[0];
                for (int r = 1; r < csize; ++r) {
                    t.sum_a += sh.fin[r].sum_a;
                    t.sum_ayfy += sh.fin[r].sum_ayfy;
                    t.sum_f0 += sh.fin[r].sum_f0;
                    t.n0 += sh.fin[r].n0;
                    t.nsv += sh.fin[r].nsv;
                }
                BatchResultDev R;
                R.b_up = up.f;
                R.b_low = low.f;
                R.b = t.n0 > 0 ? t.sum_f0 / (double)t.n0 : 0.5 * (up.f + low.f);
                R.objective = t.sum_a - 0.5 * t.sum_ayfy;
                R.iters = iter;
                R.status = status_code;
                R.n_sv = (int32_t)t.nsv;
                B.results[job] = R;
                if (B.done) {
                    __threadfence_system();
                    st_release_sys_i32(B.done + job, 1);
                }
            }
            cluster.sync();   // shared memory of the cluster is reused by the next job
        }
    }
    cluster.sync();
}

template <int MODE>
void *batch_kernel_for(int lpr)
{
    switch (lpr) {
    case 1: return (void *)smo_batch_kernel<MODE, 1>;
    case 2: return (void *)smo_batch_kernel<MODE, 2>;
    case 4: return (void *)smo_batch_kernel<MODE, 4>;
    case 8: return (void *)smo_batch_kernel<MODE, 8>;
    case 16: return (void *)smo_batch_kernel<MODE, 16>;
    case 32: return (void *)smo_batch_kernel<MODE, 32>;
    default: return nullptr;
    }
}

void *batch_fn(int mode, int lpr)
{
    if (mode == MODE_MIXED) return batch_kernel_for<MODE_MIXED>(lpr);
    if (mode == MODE_FP64) return batch_kernel_for<MODE_FP64>(lpr);
    if (mode == MODE_BINARY) return batch_kernel_for<MODE_BINARY>(lpr);
    return nullptr;
}

}  // namespace
}  // namespace smo

size_t smo_batch_smem(int mode, int d, int ktab_len, int maxnnz)
{
    // mixed mode: each warp's target fragments of the tensor-core row tiles
    return smo_layout(mode, d, ktab_len, maxnnz, 0, 0, 0).total + (mode == MODE_MIXED ? smo::kFragBytes : 0);
}

int smo_batch_max_clusters(int mode, int lpr, int dense, size_t smem, int cs)
{
    (void)dense;
    void *fn = smo::batch_fn(mode, lpr);
    if (!fn) return 0;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
    if (cs > 1 && cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) return 0;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = (unsigned)cs;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cudaLaunchConfig_t q = {};
    q.gridDim = dim3(cs);
    q.blockDim = dim3(smo::kThreads);
    q.dynamicSmemBytes = smem;
    q.attrs = &attr;
    q.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, fn, &q) != cudaSuccess) return 0;
    return n;
}

cudaError_t launch_smo_batch(int mode, int lpr, int dense, const BatchArgs &a, size_t smem, int cs,
                             int nclusters, cudaStream_t st)
{
    (void)dense;
    void *fn = smo::batch_fn(mode, lpr);
    if (!fn || cs < 1 || cs > smo::kMaxCluster || nclusters < 1) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (cs > 8) {
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    BatchArgs args = a;
    void *params[] = {&args};
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = (unsigned)cs;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(cs * nclusters));
    cfg.blockDim = dim3(smo::kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, fn, params);
}

}  // namespace svmgb
