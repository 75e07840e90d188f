// sic_kernels.cu -- sm_103a kernels of the SIC step.
//
//  K1 k_push_deposit  fused gather -> kick -> drift -> deposit over work items
//                     (consecutive tracers of one sheet); the whole mesh of the
//                     current simulation is staged in shared memory as an int64
//                     histogram and flushed to HBM with int64 atomics.
//  K2 k_field         per simulation: deposit the item seams, exact integer
//                     prefix sum of the mesh, neutralising mean and zero-mean
//                     field with one final rounding, field energy, history row.
//
// Deposit (Sec. 2.3, Eq. overlap and Eq. rho_sum): the particle between two
// tracers spreads its charge Q_s uniformly over [a, b]; cell j receives
// Q_s |[a, b] ∩ cell j| / (b - a).  In fixed point the cumulative charge at
// each interior cell edge e_k is C_k = round(Q_s (e_k - a) / (b - a)) and
// cell k receives C_k - C_{k-1} (C_0 = 0, C_last = Q_s), so the pieces of a
// segment always sum to Q_s exactly and the mesh is independent of the order
// in which the integer atomics land.
#include <cuda_runtime.h>
#include <stdint.h>

#include "sic_internal.h"

namespace sic {

namespace {

__device__ __forceinline__ int cell_of(long long u) { return (int)(u >> 32); }
__device__ __forceinline__ unsigned frac_of(long long u) { return (unsigned)(unsigned long long)u; }

// floor-mod of a cell number into [0, nx) for |c| < 2^30
__device__ __forceinline__ int wrap_cell(int c, const NxDiv &d)
{
    unsigned n = (unsigned)c + (unsigned)d.offset;
    unsigned t = __umulhi(d.magic, n);
    unsigned q = (t + ((n - t) >> 1)) >> d.shift;
    return (int)(n - q * (unsigned)d.nx);
}

// Per-thread run of consecutive contributions to one cell; a cell change
// commits the run with one shared-memory int64 atomic.
struct RunAcc {
    unsigned long long *h;
    int cell;
    long long sum;
    __device__ __forceinline__ explicit RunAcc(unsigned long long *hist) : h(hist), cell(-1), sum(0) {}
    __device__ __forceinline__ void add(int j, long long v)
    {
        if (j == cell) {
            sum += v;
            return;
        }
        if (sum)
            atomicAdd(h + cell, (unsigned long long)sum);
        cell = j;
        sum = v;
    }
    __device__ __forceinline__ void flush()
    {
        if (sum)
            atomicAdd(h + cell, (unsigned long long)sum);
        sum = 0;
        cell = -1;
    }
};

// Deposit one segment between fixed-point positions ua (cell ja mod nx) and
// ub (cell jb mod nx) carrying q units; returns its length in 2^-32 cells.
// Up to two box lengths the cumulative cut points are walked edge by edge;
// a longer segment (it wraps the box, or its tracers left the valid range)
// takes a bounded O(nx) path: the overlap of each cell summed over all its
// images, one rounding per cell, the remainder on the first interior cell.
__device__ __forceinline__ long long emit_segment(long long ua, int ja, long long ub, int jb, int q,
                                                  int nx, RunAcc &acc)
{
    if (ub < ua) {
        const long long t = ua;
        ua = ub;
        ub = t;
        const int tj = ja;
        ja = jb;
        jb = tj;
    }
    const int ca = cell_of(ua), cb = cell_of(ub);
    const long long span = ub - ua;
    if (ca == cb) {  // also the zero-length segment: all charge in the cell holding it
        acc.add(ja, q);
        return span;
    }
    const float inv = __frcp_rn(__ll2float_rn(span));
    const float qf = __int2float_rn(q);
    const long long ncut = (long long)cb - (long long)ca;
    if (ncut <= 2LL * nx) {
        long long d = (1LL << 32) - (long long)frac_of(ua);  // a to the first interior edge
        int prev = 0;
        int j = ja;
        for (int k = 0; k < (int)ncut; ++k) {
            const float t = __fmul_rn(__ll2float_rn(d), inv);
            int c = __float2int_rn(__fmul_rn(t, qf));
            c = min(max(c, prev), q);
            acc.add(j, (long long)(c - prev));
            prev = c;
            j = (j + 1 == nx) ? 0 : j + 1;
            d += (1LL << 32);
        }
        acc.add(j, (long long)(q - prev));
        return span;
    }
    const long long nint = ncut - 1;  // whole cells strictly inside (a, b)
    const int jfix = (ja + 1 == nx) ? 0 : ja + 1;
    long long given = 0;
    for (int j = 0; j < nx; ++j) {
        int o = j - jfix;
        o += (o < 0) ? nx : 0;
        const long long cnt = (nint > o) ? (nint - o - 1) / nx + 1 : 0;
        long long ov = cnt << 32;
        if (j == ja)
            ov += (1LL << 32) - (long long)frac_of(ua);
        if (j == jb)
            ov += (long long)frac_of(ub);
        int pc = __float2int_rn(__fmul_rn(__fmul_rn(__ll2float_rn(ov), inv), qf));
        pc = min(max(pc, 0), q);
        if (j != jfix) {
            given += pc;
            acc.add(j, (long long)pc);
        }
    }
    // jfix holds at least one whole image: give it the rest so the pieces sum to q
    acc.add(jfix, (long long)q - given);
    return span;
}

struct K1Shared {
    long long fu[2][SIC_K1_BLOCK];  // first tracer of each thread (new position)
    int fj[2][SIC_K1_BLOCK];        // its cell mod nx
    int fq[2][SIC_K1_BLOCK];        // its half charge
    long long pu[2];                // last tracer of the previous tile of the item
    int pj[2];
    int pq[2];
    double ra[SIC_K1_BLOCK / 32];
    double rb[SIC_K1_BLOCK / 32];
    long long rm[SIC_K1_BLOCK / 32];
};

#define K1_FIXED_BYTES ((sizeof(K1Shared) + 15) / 16 * 16)

template <bool PUSH, bool DEPOSIT, bool PER_Q>
__global__ void __launch_bounds__(SIC_K1_BLOCK, 2)
    k_push_deposit(const SimDev *__restrict__ sims, const WorkItem *__restrict__ items,
                   const int32_t *__restrict__ cta_begin, int nx_max, float kick_scale, int drift)
{
    constexpr int B = SIC_K1_BLOCK, R = SIC_K1_R, TILE = SIC_K1_TILE;
    extern __shared__ __align__(16) unsigned char smem[];
    K1Shared &sh = *reinterpret_cast<K1Shared *>(smem);
    unsigned long long *hist = reinterpret_cast<unsigned long long *>(smem + K1_FIXED_BYTES);
    float2 *ek = reinterpret_cast<float2 *>(hist + nx_max);

    const int tid = threadIdx.x;
    const int ib = cta_begin[blockIdx.x], ie = cta_begin[blockIdx.x + 1];
    int cur = -1, nx = 0, parity = 0;
    long long *U = nullptr;
    float *V = nullptr;
    const int32_t *Qh = nullptr;
    unsigned long long *mesh = nullptr;
    int64_t *edge_first = nullptr, *edge_last = nullptr;
    ItemDiag *idiag = nullptr;
    SimScalars *sc = nullptr;
    NxDiv dv{};
    bool range_err = false;

    for (int it = ib; it < ie; ++it) {
        const WorkItem W = items[it];
        if (W.sim != cur) {
            if (DEPOSIT && cur >= 0) {
                __syncthreads();
                for (int j = tid; j < nx; j += B) {
                    const unsigned long long h = hist[j];
                    if (h)
                        atomicAdd(mesh + j, h);
                }
            }
            if (range_err && sc) {
                atomicOr(&sc->err, SIC_ERR_RANGE);
                range_err = false;
            }
            __syncthreads();
            cur = W.sim;
            const SimDev &S = sims[cur];
            U = reinterpret_cast<long long *>(S.U);
            V = S.V;
            Qh = S.Qh;
            mesh = S.mesh;
            edge_first = S.edge_first;
            edge_last = S.edge_last;
            idiag = S.item_diag;
            sc = S.sc;
            dv = S.div;
            nx = dv.nx;
            if (DEPOSIT)
                for (int j = tid; j < nx; j += B)
                    hist[j] = 0ull;
            if (PUSH)
                for (int j = tid; j < nx; j += B)
                    ek[j] = S.Ek[j];
            __syncthreads();
        }

        const int qs_uniform = 2 * W.qh;
        const float qh_uniform = (float)W.qh;
        float acc_a = 0.f, acc_b = 0.f;
        long long maxseg = 0;
        const int ntile = (W.count + TILE - 1) / TILE;
        for (int tl = 0; tl < ntile; ++tl, parity ^= 1) {
            const long long base = W.t0 + (long long)tl * TILE;
            const int m = min(TILE, W.count - tl * TILE);
            const int l0 = tid * R;
            const int rn = max(0, min(R, m - l0));
            long long u[R];
            float v[R];
            int q[R];
            int jn[R];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                u[r] = 0;
                v[r] = 0.f;
                q[r] = 0;
                jn[r] = 0;
            }
            if (rn == R) {
                const longlong2 *pu = reinterpret_cast<const longlong2 *>(U + base + l0);
#pragma unroll
                for (int k = 0; k < R / 2; ++k) {
                    const longlong2 t = pu[k];
                    u[2 * k] = t.x;
                    u[2 * k + 1] = t.y;
                }
                if (PUSH) {
                    const float4 *pv = reinterpret_cast<const float4 *>(V + base + l0);
#pragma unroll
                    for (int k = 0; k < R / 4; ++k) {
                        const float4 t = pv[k];
                        v[4 * k] = t.x;
                        v[4 * k + 1] = t.y;
                        v[4 * k + 2] = t.z;
                        v[4 * k + 3] = t.w;
                    }
                }
                if (PER_Q) {
                    const int4 *pq = reinterpret_cast<const int4 *>(Qh + base + l0);
#pragma unroll
                    for (int k = 0; k < R / 4; ++k) {
                        const int4 t = pq[k];
                        q[4 * k] = t.x;
                        q[4 * k + 1] = t.y;
                        q[4 * k + 2] = t.z;
                        q[4 * k + 3] = t.w;
                    }
                }
            } else {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    if (r < rn) {
                        u[r] = U[base + l0 + r];
                        if (PUSH)
                            v[r] = V[base + l0 + r];
                        if (PER_Q)
                            q[r] = Qh[base + l0 + r];
                    }
                }
            }

            // gather (linear weighting), kick, drift
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (r < rn) {
                    const int c = cell_of(u[r]);
                    int j = wrap_cell(c, dv);
                    if (PUSH) {
                        const float f = __uint2float_rn(frac_of(u[r])) * 2.3283064365386963e-10f;
                        const float2 e = ek[j];
                        const float a = fmaf(f, e.y, e.x);
                        const float vo = v[r];
                        const float vn = fmaf(kick_scale, a, vo);
                        const float qq = PER_Q ? (float)q[r] : qh_uniform;
                        acc_a = fmaf(qq, fmaf(vo, vo, vn * vn), acc_a);
                        acc_b = fmaf(qq, vo + vn, acc_b);
                        v[r] = vn;
                        if (drift) {
                            const long long nu = u[r] + __float2ll_rn(vn * 4294967296.0f);
                            const int cn = cell_of(nu);
                            const int dc = cn - c;
                            if (dc >= -nx && dc < nx) {
                                int t = j + dc;
                                t += (t < 0) ? nx : 0;
                                t -= (t >= nx) ? nx : 0;
                                j = t;
                            } else {
                                j = wrap_cell(cn, dv);
                            }
                            if ((unsigned)(cn + (1 << 30)) >= (1u << 31))
                                range_err = true;
                            u[r] = nu;
                        }
                    }
                    jn[r] = j;
                }
            }

            if (PUSH) {
                if (rn == R) {
                    if (drift) {
                        longlong2 *pu = reinterpret_cast<longlong2 *>(U + base + l0);
#pragma unroll
                        for (int k = 0; k < R / 2; ++k)
                            pu[k] = make_longlong2(u[2 * k], u[2 * k + 1]);
                    }
                    float4 *pv = reinterpret_cast<float4 *>(V + base + l0);
#pragma unroll
                    for (int k = 0; k < R / 4; ++k)
                        pv[k] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
                } else {
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        if (r < rn) {
                            if (drift)
                                U[base + l0 + r] = u[r];
                            V[base + l0 + r] = v[r];
                        }
                    }
                }
            }

            if (DEPOSIT) {
                if (rn > 0) {
                    sh.fu[parity][tid] = u[0];
                    sh.fj[parity][tid] = jn[0];
                    sh.fq[parity][tid] = q[0];
                }
                if (tl == 0 && tid == 0)
                    edge_first[W.local] = u[0];
                __syncthreads();
                RunAcc acc(hist);
                if (tid == 0 && tl > 0) {
                    const int qs = PER_Q ? sh.pq[parity ^ 1] + q[0] : qs_uniform;
                    const long long sp =
                        emit_segment(sh.pu[parity ^ 1], sh.pj[parity ^ 1], u[0], jn[0], qs, nx, acc);
                    maxseg = max(maxseg, sp);
                }
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    if (r < rn) {
                        const int l = l0 + r;
                        if (l + 1 < m) {
                            long long ub;
                            int jb, qb;
                            if (r + 1 < R) {
                                ub = u[r + 1];
                                jb = jn[r + 1];
                                qb = q[r + 1];
                            } else {
                                ub = sh.fu[parity][tid + 1];
                                jb = sh.fj[parity][tid + 1];
                                qb = sh.fq[parity][tid + 1];
                            }
                            const int qs = PER_Q ? q[r] + qb : qs_uniform;
                            const long long sp = emit_segment(u[r], jn[r], ub, jb, qs, nx, acc);
                            maxseg = max(maxseg, sp);
                        } else if (tl + 1 < ntile) {
                            sh.pu[parity] = u[r];
                            sh.pj[parity] = jn[r];
                            sh.pq[parity] = q[r];
                        } else {
                            edge_last[W.local] = u[r];
                        }
                    }
                }
                acc.flush();
            }
        }

        // per-item diagnostics, reduced in a fixed order
        double da = acc_a, db = acc_b;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            da += __shfl_down_sync(0xffffffffu, da, o);
            db += __shfl_down_sync(0xffffffffu, db, o);
            maxseg = max(maxseg, __shfl_down_sync(0xffffffffu, maxseg, o));
        }
        if ((tid & 31) == 0) {
            sh.ra[tid >> 5] = da;
            sh.rb[tid >> 5] = db;
            sh.rm[tid >> 5] = maxseg;
        }
        __syncthreads();
        if (tid == 0) {
            ItemDiag d;
            d.ke = 0.0;
            d.p = 0.0;
            d.maxseg = 0;
            d.pad = 0;
            for (int w = 0; w < B / 32; ++w) {
                d.ke += sh.ra[w];
                d.p += sh.rb[w];
                d.maxseg = max((long long)d.maxseg, sh.rm[w]);
            }
            idiag[W.local] = d;
        }
        __syncthreads();
    }
    if (DEPOSIT && cur >= 0) {
        __syncthreads();
        for (int j = tid; j < nx; j += B) {
            const unsigned long long h = hist[j];
            if (h)
                atomicAdd(mesh + j, h);
        }
    }
    if (range_err && sc)
        atomicOr(&sc->err, SIC_ERR_RANGE);
}

// ---------------------------------------------------------------- K2 ----

__device__ __forceinline__ double i128_to_double(__int128 v)
{
    const long long hi = (long long)(v >> 64);
    const unsigned long long lo = (unsigned long long)v;
    return __fma_rn((double)hi, 18446744073709551616.0, __ull2double_rn(lo));
}

__device__ __forceinline__ __int128 shfl_down_i128(__int128 v, int o)
{
    long long lo = (long long)(unsigned long long)v;
    long long hi = (long long)(v >> 64);
    lo = __shfl_down_sync(0xffffffffu, lo, o);
    hi = __shfl_down_sync(0xffffffffu, hi, o);
    return (__int128)(((unsigned __int128)(unsigned long long)hi << 64) | (unsigned long long)lo);
}

constexpr int K2_PER_MAX = (SIC_NX_MAX + SIC_K2_BLOCK - 1) / SIC_K2_BLOCK;

__global__ void __launch_bounds__(SIC_K2_BLOCK)
    k_field(const SimDev *__restrict__ sims, const FieldJob *__restrict__ jobs, int nx_max, int record)
{
    constexpr int B = SIC_K2_BLOCK, NW = B / 32;
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned long long *sm = reinterpret_cast<unsigned long long *>(smem);
    float *sE = reinterpret_cast<float *>(sm + nx_max);
    __shared__ long long s_w[NW];
    __shared__ long long s_hi[NW], s_lo[NW];
    __shared__ double s_a[NW], s_b[NW], s_c[NW];
    __shared__ long long s_m[NW];
    __shared__ long long s_sumD_hi, s_sumD_lo;
    __shared__ double s_we, s_ke, s_p;
    __shared__ long long s_maxseg;

    const SimDev &S = sims[jobs[blockIdx.x].slot];
    const int nx = S.div.nx;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    for (int j = tid; j < nx; j += B) {
        sm[j] = S.mesh[j];
        S.mesh[j] = 0ull;
    }
    __syncthreads();

    // seams: the last segment of every item, whose far tracer another item moved
    long long maxseg = 0;
    {
        RunAcc acc(sm);
        for (int k = tid; k < S.n_items; k += B) {
            const WorkItem W = S.items[k];
            if (W.seam_next < 0)
                continue;
            const WorkItem Wn = S.items[W.seam_next];
            const long long ua = S.edge_last[k];
            const long long ub = S.edge_first[W.seam_next] + W.seam_shift;
            const int qs = S.Qh ? S.Qh[W.t0 + W.count - 1] + S.Qh[Wn.t0] : W.qh + Wn.qh;
            const int ja = wrap_cell(cell_of(ua), S.div);
            const int jb = wrap_cell(cell_of(ub), S.div);
            const long long sp = emit_segment(ua, ja, ub, jb, qs, nx, acc);
            maxseg = max(maxseg, sp);
        }
        acc.flush();
    }
    // longest segment over the items as well
    for (int k = tid; k < S.n_items; k += B)
        maxseg = max(maxseg, (long long)S.item_diag[k].maxseg);
    __syncthreads();

    // exact prefix sums P_j = sum_{i<j} mesh_i over each thread's run of cells
    const int per = (nx + B - 1) / B;
    const int j0 = tid * per;
    long long loc[K2_PER_MAX];
    long long lsum = 0;
#pragma unroll
    for (int k = 0; k < K2_PER_MAX; ++k) {
        const int j = j0 + k;
        const long long mv = (k < per && j < nx) ? (long long)sm[j] : 0;
        loc[k] = mv;
        lsum += mv;
    }
    long long incl = lsum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o)
            incl += t;
    }
    if (lane == 31)
        s_w[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        long long wv = lane < NW ? s_w[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long t = __shfl_up_sync(0xffffffffu, wv, o);
            if (lane >= o)
                wv += t;
        }
        if (lane < NW)
            s_w[lane] = wv;
    }
    __syncthreads();
    const long long qtot = s_w[NW - 1];
    const long long run0 = incl - lsum + (warp > 0 ? s_w[warp - 1] : 0);

    // D_j = nx P_j - j Q  (= nx sigma E'_j, exact) and its sum over the mesh
    __int128 dsum = 0;
    {
        long long run = run0;
#pragma unroll
        for (int k = 0; k < K2_PER_MAX; ++k) {
            const int j = j0 + k;
            if (k < per && j < nx) {
                dsum += (__int128)nx * run - (__int128)j * qtot;
                run += loc[k];
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        dsum += shfl_down_i128(dsum, o);
    if (lane == 0) {
        s_hi[warp] = (long long)(dsum >> 64);
        s_lo[warp] = (long long)(unsigned long long)dsum;
    }
    __syncthreads();
    if (tid == 0) {
        __int128 t = 0;
        for (int w = 0; w < NW; ++w)
            t += (__int128)(((unsigned __int128)(unsigned long long)s_hi[w] << 64) |
                            (unsigned long long)s_lo[w]);
        s_sumD_hi = (long long)(t >> 64);
        s_sumD_lo = (long long)(unsigned long long)t;
    }
    __syncthreads();
    const __int128 sumD = (__int128)(((unsigned __int128)(unsigned long long)s_sumD_hi << 64) |
                                     (unsigned long long)s_sumD_lo);

    // K_j = nx D_j - sum D = nx^2 sigma E_j: one rounding to double, one to float
    double wloc = 0.0;
    {
        long long run = run0;
#pragma unroll
        for (int k = 0; k < K2_PER_MAX; ++k) {
            const int j = j0 + k;
            if (k < per && j < nx) {
                const __int128 d = (__int128)nx * run - (__int128)j * qtot;
                const double kd = i128_to_double((__int128)nx * d - sumD);
                const double e = kd * S.E_scale;
                S.E64[j] = e;
                S.mesh_last[j] = loc[k];
                S.rho64[j] = i128_to_double((__int128)nx * loc[k] - qtot) * S.rho_scale;
                sE[j] = (float)(kd * S.e_scale);
                wloc += e * e;
                run += loc[k];
            }
        }
    }
    double ka = 0.0, pb = 0.0;
    if (record) {
        for (int k = tid; k < S.n_items; k += B) {
            ka += S.item_diag[k].ke;
            pb += S.item_diag[k].p;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        wloc += __shfl_down_sync(0xffffffffu, wloc, o);
        ka += __shfl_down_sync(0xffffffffu, ka, o);
        pb += __shfl_down_sync(0xffffffffu, pb, o);
        maxseg = max(maxseg, __shfl_down_sync(0xffffffffu, maxseg, o));
    }
    if (lane == 0) {
        s_a[warp] = wloc;
        s_b[warp] = ka;
        s_m[warp] = maxseg;
        s_hi[warp] = 0;
    }
    if (lane == 0)
        s_c[warp] = pb;
    __syncthreads();
    if (tid == 0) {
        double w = 0.0, kk = 0.0, pp = 0.0;
        long long mm = 0;
        for (int i = 0; i < NW; ++i) {
            w += s_a[i];
            kk += s_b[i];
            pp += s_c[i];
            mm = max(mm, s_m[i]);
        }
        s_we = w * S.half_dx;
        s_ke = kk;
        s_p = pp;
        s_maxseg = mm;
    }
    __syncthreads();
    for (int j = tid; j < nx; j += B) {
        const int j1 = (j + 1 == nx) ? 0 : j + 1;
        S.Ek[j] = make_float2(sE[j], sE[j1] - sE[j]);
    }
    if (tid == 0) {
        SimScalars *sc = S.sc;
        if (record) {
            const long long step = sc->step;
            double *row = S.hist + 4 * (step % S.hist_len);
            row[0] = sc->we;
            row[1] = S.ke_scale * s_ke;
            row[2] = S.p_scale * s_p;
            row[3] = (double)sc->q_total;
            sc->step = step + 1;
        }
        sc->we = s_we;
        sc->q_total = qtot;
        sc->maxseg = s_maxseg;
        if (S.strict && s_maxseg > ((long long)nx << 32))
            sc->err |= SIC_ERR_SEGLONG;
    }
}

__global__ void k_expand_horizontal(int64_t *U, float *V, const int64_t *ut, int32_t n, const float *vs,
                                    const int64_t *off, int32_t M)
{
    const long long total = (long long)M * n;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total;
         g += (long long)gridDim.x * blockDim.x) {
        const int s = (int)(g / n);
        const int i = (int)(g - (long long)s * n);
        U[off[s] + i] = ut[i];
        V[off[s] + i] = vs[s];
    }
}

template <bool P, bool D, bool Q>
cudaError_t prep_k1(size_t smem)
{
    static size_t done = 0;
    if (smem > done) {
        cudaError_t e = cudaFuncSetAttribute(k_push_deposit<P, D, Q>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess)
            return e;
        done = smem;
    }
    return cudaSuccess;
}

template <bool P, bool D, bool Q>
cudaError_t run_k1(const SimDev *sims, const WorkItem *items, const int32_t *cta, int grid, int nx_max,
                   float ks, int drift, cudaStream_t s)
{
    const size_t smem = k1_smem_bytes(nx_max);
    cudaError_t e = prep_k1<P, D, Q>(smem);
    if (e != cudaSuccess)
        return e;
    k_push_deposit<P, D, Q><<<grid, SIC_K1_BLOCK, smem, s>>>(sims, items, cta, nx_max, ks, drift);
    count_launches(1);
    return cudaGetLastError();
}

template <bool P, bool D, bool Q>
int occ_k1(int nx_max)
{
    const size_t smem = k1_smem_bytes(nx_max);
    if (prep_k1<P, D, Q>(smem) != cudaSuccess)
        return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_push_deposit<P, D, Q>, SIC_K1_BLOCK, smem) !=
        cudaSuccess)
        return 0;
    return n;
}

}  // namespace

size_t k1_smem_bytes(int nx_max) { return K1_FIXED_BYTES + (size_t)16 * nx_max; }

static long long g_launches = 0;
void count_launches(int64_t n) { __atomic_add_fetch(&g_launches, n, __ATOMIC_RELAXED); }
int64_t launches() { return __atomic_load_n(&g_launches, __ATOMIC_RELAXED); }

cudaError_t launch_push_deposit(const SimDev *sims, const WorkItem *items, const int32_t *cta_begin, int grid,
                                int nx_max, bool push, bool deposit, bool per_q, float kick_scale, int drift,
                                cudaStream_t s)
{
    if (push && deposit)
        return per_q ? run_k1<true, true, true>(sims, items, cta_begin, grid, nx_max, kick_scale, drift, s)
                     : run_k1<true, true, false>(sims, items, cta_begin, grid, nx_max, kick_scale, drift, s);
    if (deposit)
        return per_q ? run_k1<false, true, true>(sims, items, cta_begin, grid, nx_max, kick_scale, drift, s)
                     : run_k1<false, true, false>(sims, items, cta_begin, grid, nx_max, kick_scale, drift, s);
    return per_q ? run_k1<true, false, true>(sims, items, cta_begin, grid, nx_max, kick_scale, drift, s)
                 : run_k1<true, false, false>(sims, items, cta_begin, grid, nx_max, kick_scale, drift, s);
}

int k1_blocks_per_sm(int nx_max, bool push, bool deposit, bool per_q)
{
    if (push && deposit)
        return per_q ? occ_k1<true, true, true>(nx_max) : occ_k1<true, true, false>(nx_max);
    if (deposit)
        return per_q ? occ_k1<false, true, true>(nx_max) : occ_k1<false, true, false>(nx_max);
    return per_q ? occ_k1<true, false, true>(nx_max) : occ_k1<true, false, false>(nx_max);
}

cudaError_t launch_field(const SimDev *sims, const FieldJob *jobs, int n_jobs, int nx_max, int record,
                         cudaStream_t s)
{
    const size_t smem = (size_t)12 * nx_max;
    static size_t done = 0;
    if (smem > done) {
        cudaError_t e =
            cudaFuncSetAttribute(k_field, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess)
            return e;
        done = smem;
    }
    k_field<<<n_jobs, SIC_K2_BLOCK, smem, s>>>(sims, jobs, nx_max, record);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_expand_horizontal(int64_t *U, float *V, const int64_t *u_template, int32_t n_template,
                                     const float *v_sheet, const int64_t *sheet_offset, int32_t n_sheets,
                                     cudaStream_t s)
{
    k_expand_horizontal<<<1216, 256, 0, s>>>(U, V, u_template, n_template, v_sheet, sheet_offset, n_sheets);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace sic
