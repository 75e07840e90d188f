// sic_kernels.cu -- sm_103a kernel of the SIC step.
//
// k_step runs one whole step (or one of its halves) in a single launch, over
// one or many simulations:
//   1. a block works on one simulation at a time; each of its warps claims
//      runs of work items (up to 32 R consecutive tracers of one sheet, R per
//      lane) from that simulation's cursor, gathers E at each tracer (linear
//      weighting between the two nodes), kicks, drifts, and writes the tracer
//      to the other state buffer;
//   2. it deposits the segment from each of its tracers to the next one
//      (Sec. 2.3, Eq. overlap and Eq. rho_sum) into the block's shared-memory
//      copy of the simulation's int64 charge mesh.  The tracer after the
//      warp's last one is read from the input buffer and pushed again by the
//      warp itself, so warps and blocks never wait for one another;
//   3. when the simulation has no unclaimed items left, the block adds its
//      mesh into the global mesh with int64 atomics and counts its items on
//      the simulation's ticket; the block that completes the count runs the
//      epilogue: the exact integer field solve, the field energy, the
//      diagnostic row, and the buffer swap.  The block then moves to the
//      simulation with the most unclaimed items, until none has any.
//
// Positions are 32-bit: P = x / L 2^30 modulo 2^32 (2 bits of winding).  The
// cell coordinate of a position, 32.32 fixed point with the cell in [0, nx),
// is one multiply (P 2^2) nx; a segment is the 32-bit difference of its ends'
// P times nx 2^2, so both ends are known in the frame of the lower one.
//
// Deposit arithmetic: a segment [a, b] of q units in 32.32 fixed-point cell
// coordinates gives its first cell F = round(q (e_1 - a) / (b - a)) (FP32,
// with an approximate reciprocal, clamped to [0, q]), every whole cell inside
// P = floor(q 2^32 / (b - a)) (exact integer), and the
// last cell the rest, q - F - (cells inside) P.  The pieces always sum to q
// exactly and never go negative; the integer mesh does not depend on the
// order of the atomic adds, so results are bit-identical however the work is
// split.  Whole cells inside a long segment are added through a difference
// array, so a segment costs O(1) shared-memory atomics at any length.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "sic_internal.h"

namespace sic {

namespace {

constexpr int B = SIC_K1_BLOCK;
constexpr int R = SIC_K1_R;
constexpr int NW = SIC_K1_WARPS;
constexpr int WT = SIC_K1_WARP_TRACERS;

__device__ __forceinline__ int cell_of(long long u) { return (int)(u >> 32); }
__device__ __forceinline__ unsigned frac_of(long long u) { return (unsigned)(unsigned long long)u; }

// 32.32 fixed-point cell coordinate of a position P (x / L 2^30 modulo 2^32):
// the cell in [0, nx) in the high word, the fraction of the cell in the low
// word, exactly (one 32 x 32 -> 64 multiply of the box fraction P 2^2 by nx)
__device__ __forceinline__ long long cell_coord(unsigned p, int nx)
{
    return (long long)((unsigned long long)(p << SIC_POS_WIND_BITS) * (unsigned)nx);
}

// The segment from position pa to pb in 32.32 cell units: the 32-bit
// difference of the positions (exact for segments shorter than 2 box lengths)
// times nx 2^2
__device__ __forceinline__ long long seg_span(unsigned pa, unsigned pb, int nx4)
{
    return (long long)(int)(pb - pa) * (long long)nx4;
}

// fraction of a cell in [0, 1) from the low word (its top 23 bits)
__device__ __forceinline__ float frac_float(unsigned lo)
{
    return __fsub_rn(__uint_as_float(0x3f800000u | (lo >> 9)), 1.0f);
}

// gather (linear weighting between nodes j and j+1), kick, drift; j is the
// cell of the new position on return.  ek[j] = (Ek_j, Ek_{j+1} - Ek_j).  The
// drift adds the velocity rounded to whole position units (exact integer
// arithmetic, wrapping modulo 4 box lengths); vmax keeps the largest |v|, and
// a step of half a box (2^29 units) or more is an error.
__device__ __forceinline__ void push_one(unsigned &p, float &v, int &j, const float2 *ek, int nx, float ks,
                                         int drift, float &vmax)
{
    const long long c = cell_coord(p, nx);
    j = cell_of(c);
    const float2 e = ek[j];
    const float a = __fmaf_rn(frac_float(frac_of(c)), e.y, e.x);
    const float vn = __fmaf_rn(ks, a, v);
    v = vn;
    if (drift) {
        vmax = fmaxf(vmax, fabsf(vn));
        p += (unsigned)__float2int_rn(vn);
        j = cell_of(cell_coord(p, nx));
    }
}

// The block's copy of the charge mesh: cell j holds hi[j] * 2^32 + lo[j].
// Adds use 32-bit shared-memory atomics (a carry out of the low word goes to
// the high word), which the hardware executes natively.
struct Hist {
    unsigned *lo;
    unsigned *hi;
    __device__ __forceinline__ void add(int j, long long v) const
    {
        const unsigned l = (unsigned)(unsigned long long)v;
        const unsigned h = (unsigned)((unsigned long long)v >> 32);
        const unsigned old = atomicAdd(lo + j, l);
        const unsigned c = h + ((old + l < old) ? 1u : 0u);
        if (c)
            atomicAdd(hi + j, c);
    }
    __device__ __forceinline__ unsigned long long get(int j) const
    {
        return ((unsigned long long)hi[j] << 32) | lo[j];
    }
    __device__ __forceinline__ void set(int j, unsigned long long v) const
    {
        lo[j] = (unsigned)v;
        hi[j] = (unsigned)(v >> 32);
    }
};

// Per-thread run of consecutive contributions to one cell; a cell change
// commits the run to the block's mesh.
struct RunAcc {
    Hist h;
    int cell;
    long long sum;
    __device__ __forceinline__ explicit RunAcc(const Hist &hist) : h(hist), cell(-1), sum(0) {}
    __device__ __forceinline__ void add(int j, long long v)
    {
        if (j == cell) {
            sum += v;
            return;
        }
        if (sum)
            h.add(cell, sum);
        cell = j;
        sum = v;
    }
    __device__ __forceinline__ void flush()
    {
        if (sum)
            h.add(cell, sum);
        sum = 0;
        cell = -1;
    }
};

__device__ __forceinline__ float span_to_float(long long span)
{
    if ((unsigned long long)span < (1ull << 32))
        return __uint2float_rn((unsigned)span);
    return __fmaf_rn(__int2float_rn((int)(span >> 32)), 4294967296.0f, __uint2float_rn(frac_of(span)));
}

// floor(q 2^32 / span) for 0 <= q <= 2^28 and 2^32 < span < 2^46 (a particle
// that crosses two or more cell edges): the whole-cell charge of a box
// particle.  The float estimate (relative error below 2^-20, so within 256
// of the quotient) is corrected once with the exact remainder and then by
// at most two steps each way; the result is the exact integer floor, with
// no 64-bit integer division.
__device__ __forceinline__ long long div_q32(int q, long long span)
{
    const long long num = (long long)q << 32;
    float inv;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(inv) : "f"(span_to_float(span)));
    long long P = __float2ll_rz(__fmul_rn(__fmul_rn(__int2float_rn(q), 4294967296.0f), inv));
    long long r = num - P * span;
    P += __float2ll_rn(__fmul_rn(__ll2float_rn(r), inv));
    r = num - P * span;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        if (r < 0) {
            P -= 1;
            r += span;
        } else if (r >= span) {
            P += 1;
            r -= span;
        }
    }
    return P;
}

// n whole cells starting at cell js (mod nx) each receive p units: +p at js
// and -p after the range in the block's difference array (two's complement
// in the same 32-bit lo/hi form as the mesh, so the adds are native shared
// atomics), summed into the mesh when the block leaves the simulation
__device__ __noinline__ void range_add(int js, long long n, long long p, int nx, const Hist &dh, int *diff_used)
{
    const long long full = n < nx ? 0 : n / nx;  // 0 or 1 for a particle shorter than 1.5 box lengths
    const int rem = (int)(n - full * nx);
    if (full)
        dh.add(0, full * p);
    if (rem) {
        const int e = js + rem;
        dh.add(js, p);
        if (e <= nx) {
            dh.add(e, -p);
        } else {
            dh.add(0, p);
            dh.add(e - nx, -p);
        }
    }
    *diff_used = 1;
}

// Deposit one segment that crosses at least one cell edge, between
// fixed-point positions ua (cell ja mod nx) and ub (cell jb mod nx), carrying
// q units.  maxseg tracks the longest such segment, in 2^-16 cells
// (saturating).
// Adds each piece straight into the block's mesh.
struct DirectAdd {
    Hist h;
    __device__ __forceinline__ void add(int j, long long v) const
    {
        if (v)
            h.add(j, v);
    }
};

template <class ACC>
__device__ __forceinline__ void emit_cross(long long ua, int ja, long long ub, int jb, int q, int nx, ACC &acc,
                                           const Hist &diff, int *diff_used, unsigned &maxseg)
{
    if (ub < ua) {
        const long long t = ua;
        ua = ub;
        ub = t;
        const int tj = ja;
        ja = jb;
        jb = tj;
    }
    const long long span = ub - ua;
    maxseg = max(maxseg, (unsigned)min((unsigned long long)span >> 16, 0xffffffffull));
    const unsigned la = frac_of(ua);
    const float df = la ? __uint2float_rn(0u - la) : 4294967296.0f;  // a to the first edge
    // an approximate reciprocal is enough: F is clamped to [0, q] and the
    // other end takes q - F, so the charge stays exact
    float inv;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(inv) : "f"(span_to_float(span)));
    int F = __float2int_rn(__fmul_rn(__fmul_rn(df, inv), __int2float_rn(q)));
    F = min(max(F, 0), q);
    const long long ncut = (long long)cell_of(ub) - (long long)cell_of(ua);
    if (ncut == 1) {
        acc.add(ja, F);
        acc.add(jb, q - F);
        return;
    }
    const long long nint = ncut - 1;
    const long long P = div_q32(q, span);  // span > 2^32: two or more edges
    const long long inner = nint * P;
    if ((long long)F > (long long)q - inner)
        F = (int)((long long)q - inner);
    acc.add(ja, F);
    int j = (ja + 1 == nx) ? 0 : ja + 1;
    if (nint <= 2) {
        acc.add(j, P);
        if (nint == 2) {
            j = (j + 1 == nx) ? 0 : j + 1;
            acc.add(j, P);
        }
    } else {
        range_add(j, nint, P, nx, diff, diff_used);
    }
    acc.add(jb, (long long)q - F - inner);
}

// First-order weighting of a box particle (Sec. 2.4), between 32.32 cell
// coordinates ua and ub (any order, the lower end's cell possibly outside
// [0, nx)), q units.  Its zero-order piece in each cell (the pieces of
// emit_cross: first, whole cells inside, the rest) is shared between the
// cell's two nodes by the piece's centroid: the upper node gets round(piece
// (s0 + s1) / 2) of a piece over [s0, s1] of the cell, the lower one the
// rest.  That is the hat weighting of a uniform density exactly, up to the
// rounding of each share, and the node charges sum to q.
__device__ __forceinline__ int wrap_near(int c, int nx)
{
    while (c < 0)
        c += nx;
    while (c >= nx)
        c -= nx;
    return c;
}

template <class ACC>
__device__ __forceinline__ void emit_first(long long ua, long long ub, int q, int nx, ACC &acc,
                                           const Hist &diff, int *diff_used, unsigned &maxseg)
{
    if (ub < ua) {
        const long long t = ua;
        ua = ub;
        ub = t;
    }
    const int ja = wrap_near(cell_of(ua), nx);
    const int ja1 = (ja + 1 == nx) ? 0 : ja + 1;
    const unsigned la = frac_of(ua), lb = frac_of(ub);
    const long long ncut = (long long)cell_of(ub) - (long long)cell_of(ua);
    const long long span = ub - ua;
    maxseg = max(maxseg, (unsigned)min((unsigned long long)span >> 16, 0xffffffffull));
    if (ncut == 0) {  // inside one cell (or a point): centroid (la + lb) / 2
        const long long Y =
            (long long)(((unsigned long long)q * ((unsigned long long)la + lb) + (1ull << 32)) >> 33);
        acc.add(ja, (long long)q - Y);
        acc.add(ja1, Y);
        return;
    }
    const float df = la ? __uint2float_rn(0u - la) : 4294967296.0f;  // a to the first edge
    float inv;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(inv) : "f"(span_to_float(span)));
    long long F = __float2int_rn(__fmul_rn(__fmul_rn(df, inv), __int2float_rn(q)));
    F = min(max(F, 0ll), (long long)q);
    const long long nint = ncut - 1;
    const long long P = nint > 0 ? div_q32(q, span) : 0;
    const long long inner = nint * P;
    if (F > (long long)q - inner)
        F = (long long)q - inner;
    const long long Lr = (long long)q - F - inner;  // the last cell's piece
    // shares of the upper nodes: first piece over [la, 1], whole cells 1/2,
    // last piece over [0, lb]
    const long long YF = (long long)(((unsigned long long)F * ((1ull << 32) + la) + (1ull << 32)) >> 33);
    const long long YP = (P + 1) >> 1;
    const long long YL = (long long)(((unsigned long long)Lr * lb + (1ull << 32)) >> 33);
    const int jb = wrap_near(cell_of(ub), nx);
    const int jb1 = (jb + 1 == nx) ? 0 : jb + 1;
    acc.add(ja, F - YF);
    if (nint == 0) {  // first and last cells adjacent: node ja + 1 is jb
        acc.add(jb, YF + Lr - YL);
    } else {
        acc.add(ja1, YF + P - YP);
        // nodes ja + 2 .. ja + nint get P each (the upper share of the cell
        // below and the lower share of their own)
        if (nint > 1) {
            const int js = (ja1 + 1 == nx) ? 0 : ja1 + 1;
            if (nint - 1 <= 2) {
                acc.add(js, P);
                if (nint - 1 == 2)
                    acc.add((js + 1 == nx) ? 0 : js + 1, P);
            } else {
                range_add(js, nint - 1, P, nx, diff, diff_used);
            }
        }
        acc.add(jb, YP + Lr - YL);
    }
    acc.add(jb1, YL);
}

// Piecewise-linear particles (Sec. 2.5).  The particle from ua to ub (tracers
// i, i+1) has neighbours from up (tracer i-1) and to un (tracer i+2) along
// the sheet, all in 32.32 cell coordinates, with charges qp, qs, qn.  Its
// density rho0 + g (x - c) gives, from its lower end, the cumulative charge
// qs (t + kappa t (t - 1)) at the fraction t of its length, with
// kappa = g l / (2 rho0) and g the central difference of Eq.
// gradient_rho_estimate.  The centroids are in order along the sheet exactly
// when up < ub and ua < un (or both reversed); otherwise (a fold corner), or
// when a length or the charge is zero, kappa = 0: the box particle.
__device__ __forceinline__ float pl_kappa(long long up, long long ua, long long ub, long long un, int qp, int qs,
                                          int qn)
{
    const bool inc = up < ub && ua < un, dec = up > ub && ua > un;
    const long long lp = ua > up ? ua - up : up - ua;
    const long long ls = ub > ua ? ub - ua : ua - ub;
    const long long ln = un > ub ? un - ub : ub - un;
    if (!(inc || dec) || lp == 0 || ls == 0 || ln == 0 || qs == 0)
        return 0.f;
    const float fp = __ll2float_rn(lp), fs = __ll2float_rn(ls), fn = __ll2float_rn(ln);
    const float rp = __fdiv_rn(__int2float_rn(qp), fp);
    const float rs = __fdiv_rn(__int2float_rn(qs), fs);
    const float rn = __fdiv_rn(__int2float_rn(qn), fn);
    // twice the centroid distance c_{s+1} - c_{s-1}, signed
    const float dc2 = __ll2float_rn((ub - up) + (un - ua));
    const float k = __fdiv_rn(__fmul_rn(__fsub_rn(rn, rp), fs), __fmul_rn(rs, dc2));
    return fabsf(k) < 1e30f ? k : 0.f;
}

// Deposit one piecewise-linear particle shorter than the box (at most nx
// cells, so the loop is bounded) that crosses at least one cell edge:
// the cell between the cuts k and k+1 gets round(q phi(t_{k+1})) -
// round(q phi(t_k)), phi(t) = t + kappa t (t - 1), t_k the fraction of the
// length at the k-th edge (phi(0) = 0, phi(1) = 1), so the pieces sum to q
// exactly.  A piece may be negative when |kappa| > 1 (the linear density
// changes sign inside the particle).
template <class ACC>
__device__ __forceinline__ void emit_cross_linear(long long ua, int ja, long long ub, int jb, int q, float kappa,
                                                  int nx, ACC &acc, unsigned &maxseg)
{
    if (ub < ua) {
        const long long t = ua;
        ua = ub;
        ub = t;
        const int tj = ja;
        ja = jb;
        jb = tj;
    }
    const long long span = ub - ua;
    maxseg = max(maxseg, (unsigned)min((unsigned long long)span >> 16, 0xffffffffull));
    const float inv = __frcp_rn(__ll2float_rn(span));
    const float fq = __int2float_rn(q);
    const long long ncut = (long long)cell_of(ub) - (long long)cell_of(ua);
    const long long lo = (long long)frac_of(ua);
    long long prev = 0;
    int j = ja;
    for (long long k = 1; k <= ncut; ++k) {
        const float t = __fmul_rn(__ll2float_rn((k << 32) - lo), inv);
        const float phi = __fmaf_rn(__fmul_rn(kappa, t), __fsub_rn(t, 1.0f), t);
        const long long c = __float2ll_rn(__fmul_rn(fq, phi));
        acc.add(j, c - prev);
        prev = c;
        j = (j + 1 == nx) ? 0 : j + 1;
    }
    acc.add(jb, (long long)q - prev);
}

// The same pieces as emit_cross_linear, with the particle's cells shared out
// over the 32 lanes of the warp (all lanes call it with the same particle).
template <class ACC>
__device__ __forceinline__ void emit_linear_warp(long long ua, int ja, long long ub, int jb, int q, float kappa,
                                                 int nx, ACC &acc, unsigned &maxseg, int lane)
{
    if (ub < ua) {
        const long long t = ua;
        ua = ub;
        ub = t;
        const int tj = ja;
        ja = jb;
        jb = tj;
    }
    const long long span = ub - ua;
    maxseg = max(maxseg, (unsigned)min((unsigned long long)span >> 16, 0xffffffffull));
    const float inv = __frcp_rn(__ll2float_rn(span));
    const float fq = __int2float_rn(q);
    const long long ncut = (long long)cell_of(ub) - (long long)cell_of(ua);
    const long long lo = (long long)frac_of(ua);
    auto cum = [&](long long k) -> long long {  // round(q phi(t_k)) at the k-th edge
        const float t = __fmul_rn(__ll2float_rn((k << 32) - lo), inv);
        const float phi = __fmaf_rn(__fmul_rn(kappa, t), __fsub_rn(t, 1.0f), t);
        return __float2ll_rn(__fmul_rn(fq, phi));
    };
    for (long long k0 = 0; k0 <= ncut; k0 += 32) {
        const long long k = k0 + lane;  // cell ja + k, between the edges k and k + 1
        if (k <= ncut) {
            const long long c_lo = k == 0 ? 0 : cum(k);
            const long long c_hi = k == ncut ? (long long)q : cum(k + 1);
            int j = ja + (int)k;  // k <= ncut <= nx
            if (j >= nx)
                j -= nx;
            acc.add(j, c_hi - c_lo);
        }
    }
}

// A 128-bit integer as two words (the warp's and block's fixed-point sums).
struct Acc128 {
    unsigned long long lo;
    long long hi;
};

__device__ __forceinline__ void acc_add(Acc128 &a, const Acc128 &b)
{
    const unsigned long long nlo = a.lo + b.lo;
    a.hi = a.hi + b.hi + (nlo < b.lo ? 1 : 0);
    a.lo = nlo;
}

__device__ __forceinline__ Acc128 acc_warp_sum(Acc128 a)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        Acc128 t;
        t.lo = __shfl_down_sync(0xffffffffu, a.lo, o);
        t.hi = __shfl_down_sync(0xffffffffu, a.hi, o);
        acc_add(a, t);
    }
    return a;
}

// 128-bit add into a (lo, hi) pair of 64-bit words with two atomics
__device__ __forceinline__ void atomic_add_i128(unsigned long long *lohi, __int128 v)
{
    if (v == 0)
        return;
    const unsigned long long lo = (unsigned long long)v;
    const unsigned long long hi = (unsigned long long)(v >> 64);
    const unsigned long long old = atomicAdd(lohi, lo);
    const unsigned long long carry = (old + lo < old) ? 1ull : 0ull;
    if (hi + carry)
        atomicAdd(lohi + 1, hi + carry);
}

struct Spill {
    long long a;
    unsigned err;
};

// The rare path of sum_add: the lane's sum goes into the block's 128-bit sum
// (shared memory), and so does the term y unless it fits a fresh 64-bit sum.
// y is integer-valued when it is 2^63 or more (below 2^124; inf, NaN or
// larger set bit 31 of the error word instead).
__device__ __noinline__ Spill acc_spill(long long a, float y, unsigned long long *blk)
{
    atomic_add_i128(blk, (__int128)a);
    if (fabsf(y) < 9223372036854775808.0f)
        return Spill{__float2ll_rz(y), 0u};
    const unsigned b = __float_as_uint(y);
    const int sh = (int)((b >> 23) & 0xffu) - 150;  // y = m 2^sh, sh >= 40 here
    if (sh > 100)
        return Spill{0, 0x80000000u};
    const __int128 m = (__int128)((b & 0x7fffffu) | 0x800000u) << sh;
    atomic_add_i128(blk, (b >> 31) ? -m : m);
    return Spill{0, 0u};
}

// Add y (a term already in the sum's fixed-point unit), truncated to an
// integer, to a lane's 64-bit sum.  A term of 2^62 or more, or one that
// would overflow the sum, takes the rare path, which moves the lane's sum
// into the block's 128-bit sum: the total stays exact, so it does not
// depend on the order of the additions.
__device__ __forceinline__ void sum_add(long long &a, float y, unsigned long long *blk, unsigned &err)
{
    const long long v = __float2ll_rz(y);
    const long long s = (long long)((unsigned long long)a + (unsigned long long)v);
    if (__builtin_expect(!(fabsf(y) < 4611686018427387904.0f) || ((a ^ s) & (v ^ s)) < 0, 0)) {
        const Spill r = acc_spill(a, y, blk);
        a = r.a;
        err |= r.err;
    } else {
        a = s;
    }
}

__device__ __forceinline__ double i128_words_to_double(unsigned long long lo, unsigned long long hi)
{
    return __fma_rn((double)(long long)hi, 18446744073709551616.0, __ull2double_rn(lo));
}

// ---- programmatic dependent launch: a step launched with it may start while
// the step before it in the stream finishes; it waits for that step's end
// (and its memory) before it reads anything that step writes, and lets the
// next one start once it has no more items to begin.  Without the launch
// attribute both are no-ops.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// ---- bulk-copy staging (cp.async.bulk into shared memory, mbarrier completion)

__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity)
{
    unsigned ok;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok)
                 : "r"(smem_u32(bar)), "r"(parity)
                 : "memory");
    return ok != 0;
}

// The tracer state is read once per step and is larger than L2: its copies
// are marked first to be evicted, so the kernel's code, the simulation
// tables and the meshes stay in L2 from step to step.
__device__ __forceinline__ unsigned long long l2_evict_first()
{
    unsigned long long pol;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *bar,
                                         unsigned long long pol)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
        : "memory");
}

// A bounded wait on a stage barrier: true once the phase of this parity has
// completed; false after about a second of polling (the caller raises an
// error instead of hanging).
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long *bar, unsigned parity)
{
    for (int i = 0; i < (1 << 24); ++i)
        if (mbar_try_wait(bar, parity))
            return true;
    return false;
}

constexpr int kStageBytesU = SIC_STAGE_U_BYTES;
constexpr int kStageBytesV = SIC_STAGE_V_BYTES;
constexpr int kStageBytesQ = SIC_STAGE_Q_BYTES;

// Per-warp buffer: two stages when staging (U | V | Q each), otherwise one
// scratch of new positions (U | Q) for the cross-cell pass.
template <bool PER_Q, bool STAGED>
struct WarpBuf {
    static constexpr int q_offset = STAGED ? kStageBytesU + kStageBytesV : kStageBytesU;
    static constexpr int stage = q_offset + (PER_Q ? kStageBytesQ : 0);
    static constexpr int bytes = (STAGED ? 2 : 1) * stage;
};

// Lane 0 of a warp: copy a work item's descriptor into shared memory
// without waiting for it (five 8-byte asynchronous copies, one group)
__device__ __forceinline__ void desc_fetch(WorkItem *dst, const WorkItem *src)
{
    const unsigned d = smem_u32(dst);
    unsigned long long g;
    asm("cvta.to.global.u64 %0, %1;" : "=l"(g) : "l"(src));
#pragma unroll
    for (int k = 0; k < 5; ++k)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d + 8 * k), "l"(g + 8 * k) : "memory");
    asm volatile("cp.async.commit_group;" ::: "memory");
}

__device__ __forceinline__ void desc_wait()
{
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// Lane 0 of a warp: start the bulk copies of item W (and its halo when the
// halo is the next tracer in memory) into one stage.
template <bool PER_Q>
__device__ __forceinline__ void stage_issue(const WorkItem &W, const unsigned *Uin, const float *Vin,
                                            const int32_t *Qh, char *st, unsigned long long *bar)
{
    const bool contiguous_halo = (W.halo == W.t0 + W.count);
    const int n = W.count + (contiguous_halo ? 1 : 0);
    const unsigned b = (unsigned)(n * 4 + 15) & ~15u;  // the same for positions, velocities, charges
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(bar, (PER_Q ? 3u : 2u) * b);
    const unsigned long long pol = l2_evict_first();
    bulk_g2s(st, Uin + W.t0, b, bar, pol);
    bulk_g2s(st + kStageBytesU, Vin + W.t0, b, bar, pol);
    if (PER_Q)
        bulk_g2s(st + kStageBytesU + kStageBytesV, Qh + W.t0, b, bar, pol);
}

struct Shared {
    SimDev sim;              // the current simulation's descriptor
    unsigned long long mbar[NW][2];
    struct alignas(16) Slot {
        WorkItem w;
    } desc[NW][2];  // staging: each warp's descriptors of the items in its two stages
    int diff_used;
    int last;
    unsigned pl_prev[NW];    // piecewise-linear particles: each warp's tracer before its item
    int pl_prevq[NW];
    int taken;               // items of the current simulation the block's warps took
    int pick_n[NW], pick_s[NW];  // per warp: most unclaimed items, in which slot
    unsigned long long ke[2], p[2];          // 128-bit sums of the rare path (sum_add)
    long long wke[NW][2], wp[NW][2];         // each warp's KE and P sums (lo, hi)
    unsigned wmseg[NW];                      // each warp's longest segment
    unsigned hold, buf;                      // the simulation's scalars at entry
    long long w64[NW];
    long long hi[NW], lo[NW];
    double da[NW];
    // the epilogue's inputs, read in one round trip with the mesh: the sums'
    // limbs (ke 0-3, p 4-7), the longest segment (8), and the scalars
    unsigned long long pre[9];
    long long pre_step;
    double pre_we, pre_wk;
    unsigned pre_err, pre_hold;
    float mre[NW], mim[NW];  // each warp's part of the Fourier mode sum
};

constexpr size_t kSharedHead = (sizeof(Shared) + 15) / 16 * 16;
constexpr int kWarpCuts = 8;  // piecewise-linear particles this many cells long use the whole warp

// shared head, mesh lo/hi [nx], diff [nx + 2], kick pairs [nx] (float2);
// staging starts on a 128-byte boundary (bulk copies need 16)
__host__ __device__ __forceinline__ size_t stage_offset(int nx_max)
{
    const size_t end = kSharedHead + (size_t)8 * nx_max + (size_t)8 * (nx_max + 2) + (size_t)8 * nx_max;
    return (end + 127) / 128 * 128;
}

// ------------------------------------------------------------ epilogue ----

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

__device__ __forceinline__ __int128 make_i128(long long hi, long long lo)
{
    return (__int128)(((unsigned __int128)(unsigned long long)hi << 64) | (unsigned long long)lo);
}

// v * 2^e2 as a float, without FP64: normalise |v|, keep its top 32 bits,
// round them to 24 (relative error < 2^-24 + 2^-31), then scale by 2^(...)
__device__ __forceinline__ float pow2f(int e)
{
    e = max(-126, min(127, e));
    return __uint_as_float((unsigned)(e + 127) << 23);
}

// |v| normalised to its top 32 bits t (|v| = t 2^(e - 96) up to the bits
// below them), once for several scalings
struct Norm128 {
    unsigned t;
    int e;  // 96 - leading zeros
    bool neg, zero;
};

__device__ __forceinline__ Norm128 norm128(__int128 v)
{
    Norm128 r;
    r.zero = v == 0;
    r.neg = v < 0;
    const unsigned __int128 m = r.neg ? (unsigned __int128)(-v) : (unsigned __int128)v;
    const unsigned long long hi = (unsigned long long)(m >> 64), lo = (unsigned long long)m;
    const int lz = hi ? __clzll((long long)hi) : (lo ? 64 + __clzll((long long)lo) : 0);
    r.t = (unsigned)((m << lz) >> 96);
    r.e = 96 - lz;
    return r;
}

// v 2^e2 as a float from its normalised form
__device__ __forceinline__ float norm_to_float(const Norm128 &n, int e2)
{
    if (n.zero)
        return 0.f;
    const int e = n.e + e2;  // |v| 2^e2 = t 2^e
    const int e_a = e / 2, e_b = e - e / 2;
    const float f = __fmul_rn(__fmul_rn(__uint2float_rn(n.t), pow2f(e_a)), pow2f(e_b));
    return n.neg ? -f : f;
}

__device__ __forceinline__ float i128_to_float(__int128 v, int e2) { return norm_to_float(norm128(v), e2); }

// x 2^k exactly (x 2^k a normal double or zero)
__device__ __forceinline__ double times_pow2(double x, int k)
{
    return x * __hiloint2double((1023 + k) << 20, 0);
}

// One term of the Fourier sum sum_j y_j exp(-2 pi i j k / nx) (Sec. 3.2: the
// energy in the excited mode), the phase reduced exactly to j k mod nx.
__device__ __noinline__ void mode_add(float y, int j, int k, int nx, float &re, float &im)
{
    const int idx = (int)(((long long)j * k) % nx);
    float sn, cs;
    sincospif(__fdiv_rn(__int2float_rn(2 * idx), __int2float_rn(nx)), &sn, &cs);
    re = __fmaf_rn(y, cs, re);
    im = __fmaf_rn(-y, sn, im);
}

// Field solve of one simulation (Sec. 2.1 with C = 1) by the block holding
// its last ticket: sm (nx u64) and sE (nx floats) are this block's scratch.
//   P_j = sum_{i<j} mesh_i, D_j = nx P_j - j Q (= nx sigma E'_j exactly),
//   K_j = nx D_j - sum_j D_j (= nx^2 sigma E_j, zero mean), all integers,
//   with sum_j D_j = nx (nx - 1) Q / 2 - nx sum_i i mesh_i (from
//   sum_j P_j = sum_i (nx - 1 - i) mesh_i), so it needs no pass of its own;
//   kick table Ek_j = K_j e_scale rounded once to FP32, field energy from
//   the squares of K_j 2^-60 summed in FP32 within a warp and FP64 across.
// Everything it reads from global memory (the mesh, the step's sums, the
// scalars) is requested at once, so it waits for memory once.
// The double-precision field and density for the host are recomputed from
// mesh_last on request (k_field_out), so this path has no FP64 per cell.
__device__ void field_epilogue(const SimDev &S, int record, unsigned long long *sm, float *sE, Shared &sh)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nx = S.nx;
    if (tid >= 32 && tid < 41) {
        const unsigned long long *src = tid < 36 ? &S.acc->ke[tid - 32] : tid < 40 ? &S.acc->p[tid - 36] : &S.acc->maxseg;
        sh.pre[tid - 32] = __ldcg(src);
    } else if (tid == 64) {
        sh.pre_step = __ldcg(&S.sc->step);
    } else if (tid == 65) {
        sh.pre_we = __ldcg(&S.sc->we);
    } else if (tid == 66) {
        sh.pre_err = __ldcg(&S.sc->err);
    } else if (tid == 67) {
        sh.pre_hold = __ldcg(&S.sc->hold);
    } else if (tid == 68) {
        sh.pre_wk = __ldcg(&S.sc->wk);
    }
    for (int j = tid; j < nx; j += 4 * B) {
        unsigned long long mv[4];
#pragma unroll
        for (int k = 0; k < 4; ++k)
            mv[k] = j + k * B < nx ? __ldcg(S.mesh + j + k * B) : 0ull;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (j + k * B < nx) {
                sm[j + k * B] = mv[k];
                S.mesh[j + k * B] = 0ull;
                S.mesh_last[j + k * B] = (long long)mv[k];
            }
        }
    }
    __syncthreads();
    const int per = (nx + B - 1) / B;
    const int j0 = min(tid * per, nx), j1 = min(j0 + per, nx);
    long long lsum = 0;
    __int128 m1 = 0;  // sum_j j mesh_j over this thread's cells
#pragma unroll 1
    for (int j = j0; j < j1; ++j) {
        const long long mv = (long long)sm[j];
        lsum += mv;
        m1 += (__int128)j * mv;
    }
    long long incl = lsum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o)
            incl += t;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        m1 += shfl_down_i128(m1, o);
    if (lane == 31)
        sh.w64[warp] = incl;
    if (lane == 0) {
        sh.hi[warp] = (long long)(m1 >> 64);
        sh.lo[warp] = (long long)(unsigned long long)m1;
    }
    __syncthreads();
    long long before = 0, qtot = 0;
    __int128 M1 = 0;
    for (int w = 0; w < NW; ++w) {
        if (w < warp)
            before += sh.w64[w];
        qtot += sh.w64[w];
        M1 += make_i128(sh.hi[w], sh.lo[w]);
    }
    const long long run0 = incl - lsum + before;
    const __int128 sumD = (__int128)((long long)nx * (nx - 1) / 2) * qtot - (__int128)nx * M1;

    // K from cell to cell: D_{j+1} = D_j + nx mesh_j - Q
    float wloc = 0.f;
    const int mode_k = S.mode_k;
    float mre = 0.f, mim = 0.f;  // this thread's part of sum_j K_j 2^-60 exp(-2 pi i j k / nx)
    __int128 D = (__int128)nx * run0 - (__int128)j0 * qtot;
    __int128 K = (__int128)nx * D - sumD;
    if (S.deposit == SIC_DEPOSIT_FIRST) {
        // charge on the nodes: the trapezoid rule between nodes makes the node
        // field the mean of K at j and j + 1 (K_nx = K_0), 2 E_j = K_j + K_{j+1}
#pragma unroll 1
        for (int j = j0; j < j1; ++j) {
            D += (__int128)nx * (long long)sm[j] - qtot;
            const __int128 Kn = (__int128)nx * D - sumD;
            const Norm128 n2 = norm128(K + Kn);
            sE[j] = __fmul_rn(norm_to_float(n2, S.ek_exp - 1), S.ek_mant);
            const float kn = norm_to_float(n2, -61);
            wloc = __fmaf_rn(kn, kn, wloc);
            if (mode_k)
                mode_add(kn, j, mode_k, nx, mre, mim);
            K = Kn;
        }
    } else {
#pragma unroll 2
        for (int j = j0; j < j1; ++j) {
            const Norm128 nk = norm128(K);
            sE[j] = __fmul_rn(norm_to_float(nk, S.ek_exp), S.ek_mant);
            const float kn = norm_to_float(nk, -60);
            wloc = __fmaf_rn(kn, kn, wloc);
            if (mode_k)
                mode_add(kn, j, mode_k, nx, mre, mim);
            D += (__int128)nx * (long long)sm[j] - qtot;
            K = (__int128)nx * D - sumD;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        wloc = __fadd_rn(wloc, __shfl_down_sync(0xffffffffu, wloc, o));
    if (lane == 0)
        sh.da[warp] = (double)wloc;
    if (mode_k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            mre = __fadd_rn(mre, __shfl_down_sync(0xffffffffu, mre, o));
            mim = __fadd_rn(mim, __shfl_down_sync(0xffffffffu, mim, o));
        }
        if (lane == 0) {
            sh.mre[warp] = mre;
            sh.mim[warp] = mim;
        }
    }
    __syncthreads();
    for (int j = tid; j < nx; j += B) {
        const int j1n = (j + 1 == nx) ? 0 : j + 1;
        S.Ek[j] = make_float2(sE[j], sE[j1n] - sE[j]);
    }
    // the scalars: four threads, each one chain of (slow) FP64 arithmetic
    SimScalars *sc = S.sc;
    const long long step = sh.pre_step;
    double *row = nullptr;
    long long slot = 0;
    if (record && (tid == 0 || tid == 32 || tid == 64 || tid == 128)) {
        slot = step % S.hist_len;
        row = S.hist + 4 * slot;
    }
    auto limbs = [](const unsigned long long *l) -> double {
        const unsigned __int128 u = (unsigned __int128)l[0] + ((unsigned __int128)l[1] << 32) +
                                    ((unsigned __int128)l[2] << 64) + ((unsigned __int128)l[3] << 96);
        return i128_words_to_double((unsigned long long)u, (unsigned long long)(u >> 64));
    };
    if (tid == 32 && record)
        row[1] = S.ke_scale * times_pow2(limbs(sh.pre), -S.ke_u);
    if (tid == 64 && record)
        row[2] = S.p_scale * times_pow2(limbs(sh.pre + 4), -S.p_u);
    if (tid == 96) {
        double w = 0.0;
        for (int i = 0; i < NW; ++i)
            w += sh.da[i];
        sc->we = w * S.we_scale;
    }
    if (tid == 128 && mode_k) {
        // W_k = dx / nx |E^_k|^2 (half at k = nx/2) = (2 or 1) / nx we_scale |Z|^2
        double re = 0.0, im = 0.0;
        for (int i = 0; i < NW; ++i) {
            re += (double)sh.mre[i];
            im += (double)sh.mim[i];
        }
        if (record)
            S.mhist[slot] = sh.pre_wk;
        sc->wk = (2 * mode_k == nx ? 1.0 : 2.0) / nx * S.we_scale * (re * re + im * im);
    }
    if (tid == 0) {
        SimAccum *ac = S.acc;
        const long long mm = (long long)sh.pre[8];
#pragma unroll
        for (int k = 0; k < 4; ++k)
            ac->ke[k] = ac->p[k] = 0ull;
        ac->maxseg = 0ull;
        if (record) {
            row[0] = sh.pre_we;
            row[3] = (double)qtot;
            sc->step = step + 1;
        }
        sc->q_total = qtot;
        sc->maxseg = mm;
        unsigned err = sh.pre_err, hold = sh.pre_hold;
        if (S.strict && mm > ((long long)nx << 16))
            err |= SIC_ERR_SEGLONG;
        // the position format holds a segment exactly while it is shorter than
        // 2 box lengths; one of 1.5 or more ends the run with a range error.
        // Each end moves less than half a box per step, so a segment cannot
        // get from below 1.5 box lengths to 2.5 or more (where its difference
        // would alias to less than 1.5) in one step unseen
        if (mm >= ((long long)(3 * nx) << 15))
            err |= SIC_ERR_RANGE;
        // hold the simulation (its later steps leave it as it is) when it
        // needs the host: an error, or a particle longer than the refinement
        // length (Sec. 2.6), to be split before the run goes on.  The decision
        // is the simulation's own, so it stops at the same step alone or in
        // any batch
        if (err)
            hold |= SIC_HOLD_ERROR;
        if (S.refine_seg > 0 && mm > S.refine_seg)
            hold |= SIC_HOLD_REFINE;
        if (err != sh.pre_err)
            sc->err = err;
        if (hold != sh.pre_hold)
            sc->hold = hold;
    }
}

// inclusive prefix sum of diff[0..nx) added into hist (block-wide)
__device__ void add_diff_prefix(const Hist &hist, const Hist &diff, int nx, Shared &sh)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int per = (nx + B - 1) / B;
    const int j0 = min(tid * per, nx), j1 = min(j0 + per, nx);
    long long lsum = 0;
    for (int j = j0; j < j1; ++j)
        lsum += (long long)diff.get(j);
    long long incl = lsum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o)
            incl += t;
    }
    if (lane == 31)
        sh.w64[warp] = incl;
    __syncthreads();
    long long run = incl - lsum;
    for (int w = 0; w < warp; ++w)
        run += sh.w64[w];
    for (int j = j0; j < j1; ++j) {
        run += (long long)diff.get(j);
        hist.set(j, hist.get(j) + (unsigned long long)run);
    }
    __syncthreads();
}

// ---------------------------------------------------------------- kernel ----

// One work item (up to 32 R tracers, R per lane) of the current simulation.
// FULL: the item has all 32 R tracers, so no lane needs a bounds test.
template <bool PUSH, bool DEPOSIT, bool PER_Q, bool FULL, bool STAGED, bool GEN, class MID>
__device__ __forceinline__ void do_item(const WorkItem &W, const unsigned *__restrict__ Uin,
                                        const float *__restrict__ Vin, unsigned *__restrict__ Uout,
                                        float *__restrict__ Vout, const int32_t *__restrict__ Qh,
                                        const float2 *ek, const Hist &hist, const Hist &diff,
                                        Shared &sh, int nx, float ks, int drift, unsigned &rerr,
                                        char *st, unsigned short *tasks, long long &ake, long long &ap, unsigned &mseg,
                                        const WorkItemPL *pw, int dep, int segq, bool track_all, const MID &mid)
{
    const unsigned *stU = reinterpret_cast<const unsigned *>(st);
    const float *stV = reinterpret_cast<const float *>(st + kStageBytesU);
    const int *stQ = reinterpret_cast<const int *>(st + kStageBytesU + kStageBytesV);
    const int lane = threadIdx.x & 31;
    const int nx4 = nx << SIC_POS_WIND_BITS;
    const int m = FULL ? WT : W.count;
    const long long base = W.t0;
    const int l0 = lane * R;
    const int rn = FULL ? R : max(0, min(R, m - l0));
    const int lane_last = FULL ? 31 : (m - 1) / R;

    unsigned u[R];
    float v[R];
    int q[R];
    int jn[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        u[r] = 0u;
        v[r] = 0.f;
        q[r] = W.qh;
        jn[r] = 0;
    }
    // the tracer after the item's last one (next item, or the sheet's first)
    unsigned hu = 0u;
    float hv = 0.f;
    int hq = W.qh, hj = 0;
    bool has_halo = false;
    if (DEPOSIT && lane == lane_last && W.halo >= 0) {
        has_halo = true;
        if (STAGED && W.halo == base + m) {
            hu = stU[m];
            if (PUSH)
                hv = stV[m];
            if (PER_Q)
                hq = stQ[m];
        } else {
            hu = Uin[W.halo];
            if (PUSH)
                hv = Vin[W.halo];
            if (PER_Q)
                hq = Qh[W.halo];
        }
    }
    static_assert(R % 4 == 0, "a lane's tracers load as 16-byte vectors");
    if (STAGED || FULL || rn == R) {
        // the stage holds the whole item (and garbage past its end)
        const unsigned *pu = STAGED ? stU + l0 : Uin + base + l0;
        const float *pvv = STAGED ? stV + l0 : Vin + base + l0;
        const int *pqq = STAGED ? stQ + l0 : Qh + base + l0;
#pragma unroll
        for (int k = 0; k < R / 4; ++k) {
            // from global memory (unstaged): streaming loads, first out of L2
            const uint4 t = STAGED ? reinterpret_cast<const uint4 *>(pu)[k] : __ldcs(reinterpret_cast<const uint4 *>(pu) + k);
            u[4 * k] = t.x;
            u[4 * k + 1] = t.y;
            u[4 * k + 2] = t.z;
            u[4 * k + 3] = t.w;
            if (PUSH) {
                const float4 f =
                    STAGED ? reinterpret_cast<const float4 *>(pvv)[k] : __ldcs(reinterpret_cast<const float4 *>(pvv) + k);
                v[4 * k] = f.x;
                v[4 * k + 1] = f.y;
                v[4 * k + 2] = f.z;
                v[4 * k + 3] = f.w;
            }
            if (PER_Q) {
                const int4 c = STAGED ? reinterpret_cast<const int4 *>(pqq)[k] : __ldcs(reinterpret_cast<const int4 *>(pqq) + k);
                q[4 * k] = c.x;
                q[4 * k + 1] = c.y;
                q[4 * k + 2] = c.z;
                q[4 * k + 3] = c.w;
            }
        }
    } else {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (r < rn) {
                u[r] = Uin[base + l0 + r];
                if (PUSH)
                    v[r] = Vin[base + l0 + r];
                if (PER_Q)
                    q[r] = Qh[base + l0 + r];
            }
        }
    }

    float acc_a = 0.f, acc_b = 0.f;
    if (PUSH) {
        float vmax = 0.f;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (FULL || r < rn) {
                const float vo = v[r];
                push_one(u[r], v[r], jn[r], ek, nx, ks, drift, vmax);
                const float vn = v[r];
                if (PER_Q) {
                    const float qq = __int2float_rn(q[r]);
                    acc_a = __fmaf_rn(qq, __fmaf_rn(vo, vo, __fmul_rn(vn, vn)), acc_a);
                    acc_b = __fmaf_rn(qq, __fadd_rn(vo, vn), acc_b);
                } else {
                    acc_a = __fmaf_rn(vo, vo, __fmaf_rn(vn, vn, acc_a));
                    acc_b = __fadd_rn(acc_b, __fadd_rn(vo, vn));
                }
            }
        }
        if (!(vmax < 536870912.0f))  // a step of half a box or more
            rerr |= 1u << 30;
        if (has_halo) {
            float ignore = 0.f;
            push_one(hu, hv, hj, ek, nx, ks, drift, ignore);
        }
        if (FULL || rn == R) {
#pragma unroll
            for (int k = 0; k < R / 4; ++k) {
                __stcs(reinterpret_cast<uint4 *>(Uout + base + l0) + k,
                       make_uint4(u[4 * k], u[4 * k + 1], u[4 * k + 2], u[4 * k + 3]));
                __stcs(reinterpret_cast<float4 *>(Vout + base + l0) + k,
                       make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]));
            }
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (r < rn) {
                    Uout[base + l0 + r] = u[r];
                    Vout[base + l0 + r] = v[r];
                }
            }
        }
    } else {
#pragma unroll
        for (int r = 0; r < R; ++r)
            if (FULL || r < rn)
                jn[r] = cell_of(cell_coord(u[r], nx));
        if (has_halo)
            hj = cell_of(cell_coord(hu, nx));
    }
    mid();  // staging: the next item's copies start here

    // piecewise-linear particles (pw set): the tracer before the item and the
    // one after its halo too, for the gradients of the item's first and last
    // particles (Sec. 2.5)
    unsigned pu = 0u, nu2 = 0u;
    int pq = W.qh, nq2 = W.qh;
    bool has_prev = false, has_next2 = false;
    if (GEN && DEPOSIT && pw != nullptr) {
        const long long ip = pw->prev, in2 = pw->next2;
        has_prev = ip >= 0;
        has_next2 = in2 >= 0;
        if (lane == 0 && has_prev) {
            pu = Uin[ip];
            if (PER_Q)
                pq = Qh[ip];
            if (PUSH) {
                float pv = Vin[ip];
                int pj;
                float ignore = 0.f;
                push_one(pu, pv, pj, ek, nx, ks, drift, ignore);
            }
            pu -= pw->prev_shift;
        }
        if (lane == lane_last && has_next2) {
            nu2 = Uin[in2];
            if (PER_Q)
                nq2 = Qh[in2];
            if (PUSH) {
                float nv = Vin[in2];
                int nj;
                float ignore = 0.f;
                push_one(nu2, nv, nj, ek, nx, ks, drift, ignore);
            }
            nu2 += pw->next2_shift;
        }
    }

    if (GEN && DEPOSIT && (dep == SIC_DEPOSIT_PIC_NGP || dep == SIC_DEPOSIT_PIC_CIC)) {
        // PIC comparison deposits (Sec. 2.4): every tracer a point charge of
        // 2 Qh units, in its cell (nearest grid point) or shared between the
        // two cells whose centres bracket it (cloud in cell: the second gets
        // round(Q f), f the distance past the first centre in cells)
        DirectAdd acc{hist};
        RunAcc run(hist);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (FULL || r < rn) {
                const long long Qt = 2ll * (long long)q[r];
                if (dep == SIC_DEPOSIT_PIC_NGP) {
                    run.add(jn[r], Qt);
                } else {
                    const long long pc = cell_coord(u[r], nx) - (1ll << 31);  // centres on integers
                    int j0 = cell_of(pc);                                      // -1 before the first centre
                    j0 += (j0 < 0) ? nx : 0;
                    const int j1 = (j0 + 1 == nx) ? 0 : j0 + 1;
                    const long long p1 =
                        (long long)(((unsigned long long)Qt * (unsigned long long)frac_of(pc) + (1ull << 31)) >> 32);
                    acc.add(j0, Qt - p1);
                    acc.add(j1, p1);
                }
            }
        }
        run.flush();
    } else if (DEPOSIT) {
        hu += W.halo_shift;  // closing segment: the sheet's first tracer one winding on
        // publish the new positions (and charges) of the item in shared
        // memory, so the cross-cell segments can be shared out over the warp
        unsigned *pts = reinterpret_cast<unsigned *>(st);
        int *qpts = reinterpret_cast<int *>(st + WarpBuf<PER_Q, STAGED>::q_offset);
        if (FULL || rn == R) {
#pragma unroll
            for (int k = 0; k < R / 4; ++k) {
                reinterpret_cast<uint4 *>(pts + l0)[k] = make_uint4(u[4 * k], u[4 * k + 1], u[4 * k + 2], u[4 * k + 3]);
                if (PER_Q)
                    reinterpret_cast<int4 *>(qpts + l0)[k] = make_int4(q[4 * k], q[4 * k + 1], q[4 * k + 2], q[4 * k + 3]);
            }
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r)
                if (r < rn) {
                    pts[l0 + r] = u[r];
                    if (PER_Q)
                        qpts[l0 + r] = q[r];
                }
        }
        if (lane == lane_last && has_halo) {
            pts[m] = hu;
            if (PER_Q)
                qpts[m] = hq;
        }
        if (GEN && lane == lane_last && has_next2) {
            pts[m + 1] = nu2;
            if (PER_Q)
                qpts[m + 1] = nq2;
        }
        if (GEN && lane == 0 && has_prev) {
            sh.pl_prev[threadIdx.x >> 5] = pu;
            sh.pl_prevq[threadIdx.x >> 5] = pq;
        }
        // the next tracer of each lane's last one comes from the lane above
        const unsigned nu = __shfl_down_sync(0xffffffffu, u[0], 1);
        const int nj = __shfl_down_sync(0xffffffffu, jn[0], 1);
        const int nq = __shfl_down_sync(0xffffffffu, q[0], 1);
        const int qs_sheet = 2 * W.qh;
        __syncwarp();

        if (GEN && dep == SIC_DEPOSIT_FIRST) {
            // first-order weighting (Sec. 2.4): every particle shared out to
            // nodes by emit_first, straight into the block's mesh
            DirectAdd acc{hist};
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (FULL || r < rn) {
                    unsigned ub;
                    int qb;
                    bool seg = true;
                    if (r + 1 < R && (FULL || r + 1 < rn)) {
                        ub = u[r + 1 < R ? r + 1 : r];
                        qb = q[r + 1 < R ? r + 1 : r];
                    } else if (lane < lane_last) {
                        ub = nu;
                        qb = nq;
                    } else {
                        ub = hu;
                        qb = hq;
                        seg = has_halo;
                    }
                    if (seg) {
                        const long long ua64 = cell_coord(u[r], nx);
                        emit_first(ua64, ua64 + seg_span(u[r], ub, nx4),
                                   PER_Q ? (segq ? q[r] : q[r] + qb) : qs_sheet, nx, acc, diff, &sh.diff_used,
                                   mseg);
                    }
                }
            }
        } else {
        // segments inside one cell: whole charges summed per lane into three
        // buckets for the cells c0, c0 + 1, c0 + 2 of its first tracer (a lane
        // that reaches other cells falls back to run merging); the segments
        // that cross a cell edge are marked for the second pass.  A segment
        // lies inside one cell when its two ends share a cell and it is
        // shorter than half a box (a longer one could end in the same cell
        // one box on).
        unsigned cross = 0;
        {
            const int c0 = jn[0];
            unsigned b0 = 0, b1 = 0, b2 = 0;  // charges per tracer: charge per bucket
            unsigned cnt = 0;                 // one charge per sheet: byte k counts the segments in cell c0 + k
            int nsame = 0;
            bool wide = false;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (FULL || r < rn) {
                    unsigned ub;
                    int jb, qb;
                    bool seg = true;
                    if (r + 1 < R && (FULL || r + 1 < rn)) {
                        ub = u[r + 1 < R ? r + 1 : r];
                        jb = jn[r + 1 < R ? r + 1 : r];
                        qb = q[r + 1 < R ? r + 1 : r];
                    } else if (lane < lane_last) {
                        ub = nu;
                        jb = nj;
                        qb = nq;
                    } else {
                        ub = hu;
                        jb = hj;
                        qb = hq;
                        seg = has_halo;
                    }
                    const bool shrt = (ub - u[r] + (1u << 29)) < (1u << 30);
                    const bool same = seg && shrt && jn[r] == jb;
                    const int d = jn[r] - c0;
                    if (PER_Q) {
                        const unsigned qv = (unsigned)(segq ? q[r] : q[r] + qb);
                        b0 += (same && d == 0) ? qv : 0u;
                        b1 += (same && d == 1) ? qv : 0u;
                        b2 += (same && d == 2) ? qv : 0u;
                        wide = wide || (same && (unsigned)d > 2u);
                    } else {
                        // 2^(8 d), or 0 for d outside [0, 3] (the funnel shift
                        // clamps its count at 32; a negative d is a huge count)
                        cnt += same ? __funnelshift_lc(0u, 1u, (unsigned)d << 3) : 0u;
                        nsame += same ? 1 : 0;
                    }
                    cross |= (seg && !same) ? (1u << r) : 0u;
                }
            }
            // every inside segment of the lane in one of the four bytes (the
            // bytes cannot carry: each counts at most R)
            if (!PER_Q)
                wide = ((cnt * 0x01010101u) >> 24) != (unsigned)nsame;
            if (__builtin_expect(!wide, 1)) {
                // the cells c0 + k (k <= 3) of non-empty buckets are below nx
                if (PER_Q) {
                    if (b0)
                        hist.add(c0, b0);
                    if (b1)
                        hist.add(c0 + 1, b1);
                    if (b2)
                        hist.add(c0 + 2, b2);
                } else {
                    const long long qs = qs_sheet;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const unsigned c = (cnt >> (8 * k)) & 0xffu;
                        if (c)
                            hist.add(c0 + k, (long long)c * qs);
                    }
                }
            } else {
                RunAcc acc(hist);
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    if ((FULL || r < rn) && !((cross >> r) & 1u)) {
                        int qb;
                        bool seg = true;
                        if (r + 1 < R && (FULL || r + 1 < rn)) {
                            qb = q[r + 1 < R ? r + 1 : r];
                        } else if (lane < lane_last) {
                            qb = nq;
                        } else {
                            qb = hq;
                            seg = has_halo;
                        }
                        if (seg)
                            acc.add(jn[r], PER_Q ? (segq ? q[r] : q[r] + qb) : qs_sheet);
                    }
                }
                acc.flush();
            }
        }

        // a refinement length shorter than a cell: particles inside one cell
        // count towards the longest one too (the cross-cell ones are measured
        // where they are deposited)
        if (track_all) {
            unsigned longest = 0;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (FULL || r < rn) {
                    unsigned ub;
                    bool seg = true;
                    if (r + 1 < R && (FULL || r + 1 < rn))
                        ub = u[r + 1 < R ? r + 1 : r];
                    else if (lane < lane_last)
                        ub = nu;
                    else {
                        ub = hu;
                        seg = has_halo;
                    }
                    if (seg)
                        longest = max(longest, (unsigned)abs((int)(ub - u[r])));
                }
            }
            mseg = max(mseg, (unsigned)min(((unsigned long long)longest * (unsigned)nx4) >> 16, 0xffffffffull));
        }

        // cross-cell segments of box particles, at most one per lane (the
        // usual case): each lane deposits its own
        const int cnt = __popc(cross);
        const bool boxes = !(GEN && pw != nullptr);
        if (boxes && !__any_sync(0xffffffffu, cnt > 1)) {
            if (cross) {
                const int idx = l0 + __ffs(cross) - 1;
                const unsigned pa = pts[idx], pb = pts[idx + 1];
                const long long ua = cell_coord(pa, nx);
                const long long ub = ua + seg_span(pa, pb, nx4);
                const int qs = PER_Q ? qpts[idx] + (segq ? 0 : qpts[idx + 1]) : qs_sheet;
                DirectAdd acc{hist};
                emit_cross(ua, cell_of(ua), ub, cell_of(cell_coord(pb, nx)), qs, nx, acc, diff, &sh.diff_used, mseg);
            }
            cross = 0;
        }
        // the others: compact them into a task list and let every lane take
        // one in turn; a lane's slot is the count before it, summed from one
        // ballot per bit of the per-lane counts (0..R) when there are any
        unsigned lt;
        asm("mov.u32 %0, %%lanemask_lt;" : "=r"(lt));
        const int total = (int)__reduce_add_sync(0xffffffffu, (unsigned)__popc(cross));  // tasks of the warp
        int excl = 0;
        if (total) {
#pragma unroll
            for (int bit = 0; (1 << bit) <= R; ++bit) {
                const unsigned bb = __ballot_sync(0xffffffffu, (__popc(cross) >> bit) & 1);
                excl += __popc(bb & lt) << bit;
            }
        }
        if (total) {
            int pos = excl;
#pragma unroll
            for (int r = 0; r < R; ++r) {  // predicated stores, no loop to diverge on
                if ((cross >> r) & 1u)
                    tasks[pos++] = (unsigned short)(l0 + r);
            }
            cross = 0;
            __syncwarp();
            DirectAdd acc{hist};
            // piecewise-linear particles: kappa of the particle at idx, from
            // its neighbours' positions in the frame of its own lower end ua;
            // 0 keeps it a box (no neighbour on one side, or a box length or
            // longer)
            auto kappa_of = [&](int idx, long long ua, long long ub, int qs) -> float {
                const bool hp = idx > 0 || has_prev;
                const bool hn = idx + 2 < m || (idx + 2 == m && W.halo >= 0) || (idx + 2 == m + 1 && has_next2);
                const long long len = ub > ua ? ub - ua : ua - ub;
                if (!(hp && hn && len < ((long long)nx << 32)))
                    return 0.f;
                const int w8 = threadIdx.x >> 5;
                const unsigned pp = idx > 0 ? pts[idx - 1] : sh.pl_prev[w8];
                const long long up = ua - seg_span(pp, pts[idx], nx4);
                const long long un = ub + seg_span(pts[idx + 1], pts[idx + 2], nx4);
                const int qp = PER_Q ? (idx > 0 ? qpts[idx - 1] : sh.pl_prevq[w8]) + (segq ? 0 : qpts[idx]) : qs_sheet;
                const int qn = PER_Q ? qpts[idx + 1] + (segq ? 0 : qpts[idx + 2]) : qs_sheet;
                return pl_kappa(up, ua, ub, un, qp, qs, qn);
            };
            bool any_long = false;
            for (int k = lane; k < total; k += 32) {
                const int idx = tasks[k];
                const unsigned pa = pts[idx], pb = pts[idx + 1];
                const long long ua = cell_coord(pa, nx);
                const long long ub = ua + seg_span(pa, pb, nx4);
                const int ja = cell_of(ua), jb = cell_of(cell_coord(pb, nx));
                const int qs = PER_Q ? qpts[idx] + (segq ? 0 : qpts[idx + 1]) : qs_sheet;
                const float kappa = (GEN && pw != nullptr) ? kappa_of(idx, ua, ub, qs) : 0.f;
                if (kappa == 0.f) {
                    emit_cross(ua, ja, ub, jb, qs, nx, acc, diff, &sh.diff_used, mseg);
                } else {
                    const int cuts = cell_of(ua) > cell_of(ub) ? cell_of(ua) - cell_of(ub) : cell_of(ub) - cell_of(ua);
                    if (cuts >= kWarpCuts) {
                        tasks[k] = (unsigned short)(idx | 0x8000);  // for the whole warp, below
                        any_long = true;
                    } else {
                        emit_cross_linear(ua, ja, ub, jb, qs, kappa, nx, acc, mseg);
                    }
                }
            }
            // long piecewise-linear particles: every lane takes some of the
            // particle's cells (the pieces do not depend on who computes them)
            if (GEN && pw != nullptr && __any_sync(0xffffffffu, any_long)) {
                __syncwarp();
                for (int base = 0; base < total; base += 32) {
                    const int k = base + lane;
                    unsigned bal = __ballot_sync(0xffffffffu, k < total && (tasks[k] & 0x8000));
                    while (bal) {
                        const int src = __ffs(bal) - 1;
                        bal &= bal - 1u;
                        const int idx = tasks[base + src] & 0x7fff;
                        const unsigned pa = pts[idx], pb = pts[idx + 1];
                        const long long ua = cell_coord(pa, nx);
                        const long long ub = ua + seg_span(pa, pb, nx4);
                        const int qs = PER_Q ? qpts[idx] + (segq ? 0 : qpts[idx + 1]) : qs_sheet;
                        emit_linear_warp(ua, cell_of(ua), ub, cell_of(cell_coord(pb, nx)), qs,
                                         kappa_of(idx, ua, ub, qs), nx, acc, mseg, lane);
                    }
                }
            }
        }
        }  // not first-order
        __syncwarp();  // pts and tasks are rewritten by the next item
    }

    // this lane's kinetic-energy and momentum terms (times the sheet's half
    // charge, unless the tracers carry their own, and in the sums' fixed-point
    // units), added exactly to its running sums (summed over the warp when it
    // leaves the simulation)
    if (PUSH) {
        sum_add(ake, __fmul_rn(acc_a, W.ke_mult), sh.ke, rerr);
        sum_add(ap, __fmul_rn(acc_b, W.p_mult), sh.p, rerr);
    }
}

template <bool PUSH, bool DEPOSIT, bool PER_Q, bool STAGED, bool GEN>
__global__ void __launch_bounds__(B, SIC_K1_MIN_BLOCKS) k_step(const LaunchArgs A)
{
    extern __shared__ __align__(16) unsigned char smem[];
    Shared &sh = *reinterpret_cast<Shared *>(smem);
    const int nx_max = A.nx_max;
    unsigned long long *mesh_region = reinterpret_cast<unsigned long long *>(smem + kSharedHead);
    Hist hist;
    hist.lo = reinterpret_cast<unsigned *>(mesh_region);
    hist.hi = hist.lo + nx_max;
    Hist diff;  // the difference array of long particles: nx_max + 2 cells
    diff.lo = reinterpret_cast<unsigned *>(mesh_region + nx_max);
    diff.hi = diff.lo + nx_max + 2;
    float2 *ek = reinterpret_cast<float2 *>(mesh_region + nx_max + nx_max + 2);
    char *stage_base = reinterpret_cast<char *>(smem) + stage_offset(nx_max);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const float ks = A.kick_scale;
    const int drift = (PUSH && DEPOSIT) ? 1 : A.drift;  // a full step always drifts
    char *my_stage = stage_base + (size_t)warp * WarpBuf<PER_Q, STAGED>::bytes;
    unsigned short *tasks =
        reinterpret_cast<unsigned short *>(stage_base + (size_t)NW * WarpBuf<PER_Q, STAGED>::bytes) + warp * WT;
    unsigned phase = 0;      // bit s: parity of stage s's next completion
    int s = 0;               // the stage the warp's next item lands in
    bool timed_out = false;
    if (STAGED) {
        if (tid < 2 * NW)
            mbar_init(&sh.mbar[tid >> 1][tid & 1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }

    // the first simulation: the one that holds this block's proportional
    // share of the launch's items
    int cur;
    {
        const long long target = ((2ll * blockIdx.x + 1) * (long long)A.n_items) / (2ll * gridDim.x);
        int lo = 0, hi = A.n_slots - 1;  // last slot with slot_begin <= target
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (A.slot_begin[mid] <= target)
                lo = mid;
            else
                hi = mid - 1;
        }
        cur = lo;
    }
    unsigned rerr = 0, mseg = 0;
    long long ake = 0, ap = 0;  // this lane's KE and P sums (units 2^-ke_u, 2^-p_u)
    bool first = true;          // the block's first simulation of the launch
    bool triggered = false;     // the next launch in the stream may start
    unsigned seen = 0;          // lane 0: the simulation's claim cursor as last seen
    unsigned done_old = 0;      // thread 0: blocks counted out before this one
    bool done_early = false;

    while (cur >= 0) {
        // ---- enter simulation cur: its descriptor into shared memory (the
        // launch's table does not change while it runs)
        for (int i = tid; i < (int)(sizeof(SimDev) / 4); i += B)
            reinterpret_cast<unsigned *>(&sh.sim)[i] = reinterpret_cast<const unsigned *>(A.sims + cur)[i];
        __syncthreads();
        const SimDev &S = sh.sim;
        const WorkItem *items = S.items;
        const int n_s = A.slot_begin[cur + 1] - A.slot_begin[cur];
        const int nx = S.nx;
        if (DEPOSIT) {
            for (int j = tid; j < nx; j += B) {
                hist.lo[j] = 0u;
                hist.hi[j] = 0u;
            }
            for (int j = tid; j < nx + 2; j += B) {
                diff.lo[j] = 0u;
                diff.hi[j] = 0u;
            }
        }
        if (tid == 0) {
            sh.diff_used = 0;
            sh.taken = 0;
            sh.ke[0] = sh.ke[1] = sh.p[0] = sh.p[1] = 0ull;
        }
        if (first) {
            // a launch that may start before the previous one in its stream
            // has finished waits here: everything below may be its output
            griddep_wait();
            first = false;
        }
        // one round trip: the hold and buffer words, the kick table and each
        // warp's first claim
        if (tid == 0) {
            sh.hold = *(volatile unsigned *)&S.sc->hold;
            sh.buf = *(volatile unsigned *)&S.sc->buf;
        }
        if (PUSH) {
            for (int j = tid; j < nx; j += B)
                ek[j] = S.Ek[j];
        }

        // ---- each warp claims runs of consecutive items (guided: a claim is
        // the fraction claim_q of what it saw left, at least claim_min items)
        // and streams them through its two stages.  A run's claim is made
        // when the run before the previous one ends, so its result has had a
        // whole run to arrive when it is needed.  With staging, an item's
        // descriptor is copied into shared memory while the item before it is
        // pushed, and its data copies start halfway through that item.
        unsigned *cursor = A.cursor + cur;
        const float q = A.claim_q;
        const int claim_min = max(1, A.claim_min);
        unsigned c_old = 0, c_want = 0;  // lane 0: the claim in flight
        auto claim_issue = [&]() {
            if (lane == 0) {
                const int left = n_s - (int)min(seen, (unsigned)n_s);
                c_want = left > 0 ? (unsigned)max(claim_min, (int)((float)left * q)) : 0u;
                c_old = c_want ? atomicAdd(cursor, c_want) : (unsigned)n_s;
            }
        };
        auto claim_take = [&](int &a, int &n) {  // the first use of the claim's result
            if (lane == 0)
                seen = c_old + c_want;
            const unsigned o = __shfl_sync(0xffffffffu, c_old, 0);
            const unsigned w = __shfl_sync(0xffffffffu, c_want, 0);
            a = (int)o;
            n = (int)o < n_s ? min((int)w, n_s - (int)o) : 0;
        };
        claim_issue();  // before the hold is known: a held simulation drops it
        __syncthreads();

        // a full step leaves a held simulation (set by an earlier launch's
        // epilogue, so the same for every block of this one) as it is: its
        // items are all marked claimed, so no block picks it again in this
        // launch.  An explicit deposit or push still runs.
        if (PUSH && DEPOSIT && sh.hold) {
            if (tid == 0)
                atomicAdd(cursor, (unsigned)n_s);
            __syncthreads();  // the block's own pick below sees it taken
        } else {
        const bool track_all = S.refine_seg > 0 && S.refine_seg < (1ll << 16);  // refinement below a cell
        const int src = (int)sh.buf;
        const unsigned *Uin = S.U[src];
        const float *Vin = S.V[src];
        unsigned *Uout = S.U[src ^ 1];
        float *Vout = S.V[src ^ 1];
        const int32_t *Qh = S.Qh;
        int a, n;
        claim_take(a, n);
        claim_issue();  // the next run's claim, in flight through this run
        int count = 0;
        if (STAGED) {
            if (n > 0 && !timed_out && lane == 0) {
                desc_fetch(&sh.desc[warp][s].w, items + a);
                desc_wait();
                stage_issue<PER_Q>(sh.desc[warp][s].w, Uin, Vin, Qh, my_stage + s * WarpBuf<PER_Q, true>::stage,
                                   &sh.mbar[warp][s]);
            }
            __syncwarp();
        }
        while (n > 0) {
            int na = 0, nn = 0;
            bool took = false;
            count += n;
            for (int i = a; i < a + n && !timed_out; ++i) {
                int nxt = i + 1;
                if (nxt == a + n) {
                    claim_take(na, nn);
                    claim_issue();  // the run after it, in flight through the next run
                    took = true;
                    nxt = nn > 0 ? na : -1;
                }
                if (!STAGED && lane == 0 && i + 2 < a + n) {
                    // lane 0 reads the next descriptor to start its copies:
                    // fetch the one after it into L1 now (both of its sectors),
                    // so that read does not wait on L2
                    const char *pf = reinterpret_cast<const char *>(items + i + 2);
                    asm volatile("prefetch.global.L1 [%0];" ::"l"(pf));
                    asm volatile("prefetch.global.L1 [%0];" ::"l"(pf + sizeof(WorkItem) - 1));
                }
                const WorkItem W = STAGED ? sh.desc[warp][s].w : items[i];
                const WorkItemPL *plw = (GEN && S.pl != nullptr) ? S.pl + i : nullptr;
                if (STAGED) {
                    // the next item's descriptor comes in while this one is
                    // pushed; its copies start halfway through this item
                    if (nxt >= 0 && lane == 0)
                        desc_fetch(&sh.desc[warp][s ^ 1].w, items + nxt);
                    const bool ok = mbar_wait_bounded(&sh.mbar[warp][s], (phase >> s) & 1u);
                    phase ^= 1u << s;
                    if (!__all_sync(0xffffffffu, ok)) {
                        // give up (the next item's copies have not started): only count items
                        timed_out = true;
                        if (nxt >= 0 && lane == 0)
                            desc_wait();
                        break;
                    }
                    auto mid = [&]() {
                        if (nxt >= 0 && lane == 0) {
                            desc_wait();
                            stage_issue<PER_Q>(sh.desc[warp][s ^ 1].w, Uin, Vin, Qh,
                                               my_stage + (s ^ 1) * WarpBuf<PER_Q, true>::stage, &sh.mbar[warp][s ^ 1]);
                        }
                    };
                    char *st = my_stage + s * WarpBuf<PER_Q, true>::stage;
                    if (W.count == WT)
                        do_item<PUSH, DEPOSIT, PER_Q, true, true, GEN>(W, Uin, Vin, Uout, Vout, Qh, ek, hist, diff, sh,
                                                                  nx, ks, drift, rerr, st, tasks, ake, ap, mseg, plw,
                                                                  S.deposit, S.seg_q, track_all, mid);
                    else
                        do_item<PUSH, DEPOSIT, PER_Q, false, true, GEN>(W, Uin, Vin, Uout, Vout, Qh, ek, hist, diff, sh,
                                                                   nx, ks, drift, rerr, st, tasks, ake, ap, mseg, plw,
                                                                   S.deposit, S.seg_q, track_all, mid);
                    __syncwarp();
                    s ^= 1;
                } else {
                    auto mid = []() {};
                    if (W.count == WT)
                        do_item<PUSH, DEPOSIT, PER_Q, true, false, GEN>(W, Uin, Vin, Uout, Vout, Qh, ek, hist, diff, sh,
                                                                   nx, ks, drift, rerr, my_stage, tasks, ake, ap, mseg,
                                                                   plw, S.deposit, S.seg_q, track_all, mid);
                    else
                        do_item<PUSH, DEPOSIT, PER_Q, false, false, GEN>(W, Uin, Vin, Uout, Vout, Qh, ek, hist, diff, sh,
                                                                    nx, ks, drift, rerr, my_stage, tasks, ake, ap, mseg,
                                                                    plw, S.deposit, S.seg_q, track_all, mid);
                }
            }
            if (!took) {
                claim_take(na, nn);
                claim_issue();
            }
            a = na;
            n = nn;
        }
        if (lane == 0)
            atomicAdd(&sh.taken, count);
        if (!triggered) {
            // this block has no more items to start: the next launch in the
            // stream may begin (it waits for this one's end before it reads)
            griddep_launch_dependents();
            triggered = true;
        }

        // ---- leave: fold the block's mesh and sums into the simulation's,
        // take an item ticket, run the field epilogue if it completes it
        if (PUSH) {
            const Acc128 k2 = acc_warp_sum(Acc128{(unsigned long long)ake, ake >> 63});
            const Acc128 p2 = acc_warp_sum(Acc128{(unsigned long long)ap, ap >> 63});
            if (lane == 0) {
                sh.wke[warp][0] = (long long)k2.lo;
                sh.wke[warp][1] = k2.hi;
                sh.wp[warp][0] = (long long)p2.lo;
                sh.wp[warp][1] = p2.hi;
            }
            ake = 0;
            ap = 0;
        }
        if (DEPOSIT) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
                mseg = max(mseg, __shfl_down_sync(0xffffffffu, mseg, o));
            if (lane == 0)
                sh.wmseg[warp] = mseg;
            mseg = 0;
        }
        __syncthreads();
        if (DEPOSIT) {
            if (sh.diff_used)
                add_diff_prefix(hist, diff, nx, sh);
            for (int j = tid; j < nx; j += B) {
                const unsigned long long h = hist.get(j);
                if (h)
                    atomicAdd(S.mesh + j, h);
            }
        }
        if (rerr >> 30)  // a step of half a box or more, or a sum that is not finite
            atomicOr(&S.sc->err, SIC_ERR_RANGE);
        rerr = 0;
        if (STAGED && timed_out && lane == 0)
            atomicOr(&S.sc->err, SIC_ERR_TIMEOUT);
        if (tid == 0) {
            SimAccum *ac = S.acc;
            if (PUSH) {
                // the block's 128-bit sums, added limb by limb
                Acc128 k{sh.ke[0], (long long)sh.ke[1]}, pm{sh.p[0], (long long)sh.p[1]};
                for (int w = 0; w < NW; ++w) {
                    acc_add(k, Acc128{(unsigned long long)sh.wke[w][0], sh.wke[w][1]});
                    acc_add(pm, Acc128{(unsigned long long)sh.wp[w][0], sh.wp[w][1]});
                }
                const unsigned kl[4] = {(unsigned)k.lo, (unsigned)(k.lo >> 32), (unsigned)k.hi,
                                        (unsigned)((unsigned long long)k.hi >> 32)};
                const unsigned pl[4] = {(unsigned)pm.lo, (unsigned)(pm.lo >> 32), (unsigned)pm.hi,
                                        (unsigned)((unsigned long long)pm.hi >> 32)};
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    if (kl[i])
                        atomicAdd(&ac->ke[i], (unsigned long long)kl[i]);
                    if (pl[i])
                        atomicAdd(&ac->p[i], (unsigned long long)pl[i]);
                }
            }
            if (DEPOSIT) {
                unsigned m = 0;
                for (int w = 0; w < NW; ++w)
                    m = max(m, sh.wmseg[w]);
                if (m)
                    atomicMax(&ac->maxseg, (unsigned long long)m);
            }
        }
        __threadfence();
        __syncthreads();
        if (tid == 0) {
            // only a block that took items counts them: a block whose claims
            // all came too late adds nothing, and must not read a completed
            // count as its own (that simulation's epilogue would run twice)
            const unsigned taken = (unsigned)sh.taken;
            sh.last = 0;
            if (taken) {
                const unsigned t = atomicAdd(A.tickets + cur, taken);
                sh.last = (t + taken == (unsigned)n_s) ? 1 : 0;
            }
            // a launch of one simulation: this block claims nothing more, so
            // it counts itself out now and reads the count after the epilogue
            if (A.n_slots == 1) {
                done_old = atomicAdd(A.done, 1u);
                done_early = true;
            }
        }
        __syncthreads();
        if (sh.last) {
            __threadfence();
            if (DEPOSIT)
                field_epilogue(S, A.record, mesh_region, reinterpret_cast<float *>(ek), sh);
            if (tid == 0) {
                if (PUSH)
                    S.sc->buf = (unsigned)(src ^ 1);
                if (!DEPOSIT) {  // the epilogue did not consume the sums: drop them
                    SimAccum *ac = S.acc;
                    for (int k = 0; k < 4; ++k)
                        ac->ke[k] = ac->p[k] = 0ull;
                    ac->maxseg = 0ull;
                }
                A.tickets[cur] = 0u;
            }
        }
        }  // not held

        // ---- next: the simulation with the most unclaimed items, if any
        // (a launch of one simulation has none)
        int most = 0;
        cur = -1;
        if (A.n_slots > 1) {
            int best = -1;
            for (int j = tid; j < A.n_slots; j += B) {
                const int left = (A.slot_begin[j + 1] - A.slot_begin[j]) - (int)*(volatile unsigned *)(A.cursor + j);
                if (left > most) {
                    most = left;
                    best = j;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const int m2 = __shfl_down_sync(0xffffffffu, most, o);
                const int b2 = __shfl_down_sync(0xffffffffu, best, o);
                if (m2 > most) {
                    most = m2;
                    best = b2;
                }
            }
            if (lane == 0) {
                sh.pick_n[warp] = most;
                sh.pick_s[warp] = best;
            }
            __syncthreads();
            most = 0;
            for (int w = 0; w < NW; ++w)
                if (sh.pick_n[w] > most) {
                    most = sh.pick_n[w];
                    cur = sh.pick_s[w];
                }
            if (cur >= 0)  // its cursor as the search saw it
                seen = (unsigned)(A.slot_begin[cur + 1] - A.slot_begin[cur] - most);
        }
        __syncthreads();  // the picks and the epilogue's scratch are free again
    }

    // the last block out rewinds the claim cursors for the next launch
    if (tid == 0) {
        if (!done_early) {
            __threadfence();
            done_old = atomicAdd(A.done, 1u);
        }
        sh.last = (done_old + 1 == gridDim.x) ? 1 : 0;
    }
    __syncthreads();
    if (sh.last) {
        for (int j = tid; j < A.n_slots; j += B)
            A.cursor[j] = 0u;
        if (tid == 0)
            *A.done = 0u;
    }
}

template <bool P, bool D, bool Q, bool G, bool L>
cudaError_t prep(size_t smem)
{
    static size_t done = 0;
    if (smem > done) {
        cudaError_t e = cudaFuncSetAttribute(k_step<P, D, Q, G, L>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess)
            return e;
        done = smem;
    }
    return cudaSuccess;
}

template <bool P, bool D, bool Q, bool G, bool L>
cudaError_t run(const LaunchArgs &a, int grid, cudaStream_t s)
{
    const size_t smem = step_smem_bytes(a.nx_max, G, Q);
    cudaError_t e = prep<P, D, Q, G, L>(smem);
    if (e != cudaSuccess)
        return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(B);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const cudaError_t e2 = cudaLaunchKernelEx(&cfg, k_step<P, D, Q, G, L>, a);
    count_launches(1);
    return e2 != cudaSuccess ? e2 : cudaGetLastError();
}

template <bool P, bool D, bool Q, bool G>
int occ(int nx_max)
{
    const size_t smem = step_smem_bytes(nx_max, G, Q);
    if (prep<P, D, Q, G, false>(smem) != cudaSuccess)
        return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step<P, D, Q, G, false>, B, smem) != cudaSuccess)
        return 0;
    return n;
}

// a.gen: some simulation of the launch deposits other than box particles;
// that variant handles every kind
template <bool P, bool D, bool G>
cudaError_t run_pd(const LaunchArgs &a, int grid, bool per_q, cudaStream_t s)
{
    if (a.gen)
        return per_q ? run<P, D, true, G, true>(a, grid, s) : run<P, D, false, G, true>(a, grid, s);
    return per_q ? run<P, D, true, G, false>(a, grid, s) : run<P, D, false, G, false>(a, grid, s);
}

template <bool P, bool D, bool G>
int occ_pd(int nx_max, bool per_q)
{
    return per_q ? occ<P, D, true, G>(nx_max) : occ<P, D, false, G>(nx_max);
}

// The double-precision node field E_j and density rho_j of the latest
// deposit, recomputed from its exact charge mesh (one block of 1024 threads).
// Fourier amplitudes |X^_k| = |sum_j X_j exp(-2 pi i j k / nx)| of the FP64
// density (field 0) or node field (field 1) that k_field_out wrote, one block
// per k = 0 .. nx/2, in a fixed order of additions (Sec. 3.2).
__global__ void __launch_bounds__(256) k_spectrum(const SimDev S, int field)
{
    __shared__ double s_re[8], s_im[8];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nx = S.nx, k = blockIdx.x;
    const double *X = field ? S.E64 : S.rho64;
    double re = 0.0, im = 0.0;
    for (int j = tid; j < nx; j += 256) {
        const int idx = (int)(((long long)j * k) % nx);
        double sn, cs;
        sincospi(2.0 * idx / nx, &sn, &cs);
        re = fma(X[j], cs, re);
        im = fma(-X[j], sn, im);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        re += __shfl_down_sync(0xffffffffu, re, o);
        im += __shfl_down_sync(0xffffffffu, im, o);
    }
    if (lane == 0) {
        s_re[warp] = re;
        s_im[warp] = im;
    }
    __syncthreads();
    if (tid == 0) {
        re = 0.0;
        im = 0.0;
        for (int w = 0; w < 8; ++w) {
            re += s_re[w];
            im += s_im[w];
        }
        S.spec[k] = hypot(re, im);
    }
}

__global__ void __launch_bounds__(1024) k_field_out(const SimDev S)
{
    constexpr int BB = 1024, NWW = BB / 32;
    __shared__ long long s_w[NWW];
    __shared__ long long s_hi[NWW], s_lo[NWW];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nx = S.nx;
    const int per = (nx + BB - 1) / BB;
    const int j0 = min(tid * per, nx), j1 = min(j0 + per, nx);
    long long lsum = 0;
    for (int j = j0; j < j1; ++j)
        lsum += S.mesh_last[j];
    long long incl = lsum;
    for (int o = 1; o < 32; o <<= 1) {
        const long long t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o)
            incl += t;
    }
    if (lane == 31)
        s_w[warp] = incl;
    __syncthreads();
    long long before = 0, qtot = 0;
    for (int w = 0; w < NWW; ++w) {
        if (w < warp)
            before += s_w[w];
        qtot += s_w[w];
    }
    const long long run0 = incl - lsum + before;
    __int128 dsum = 0;
    long long run = run0;
    for (int j = j0; j < j1; ++j) {
        dsum += (__int128)nx * run - (__int128)j * qtot;
        run += S.mesh_last[j];
    }
    for (int o = 16; o > 0; o >>= 1)
        dsum += shfl_down_i128(dsum, o);
    if (lane == 0) {
        s_hi[warp] = (long long)(dsum >> 64);
        s_lo[warp] = (long long)(unsigned long long)dsum;
    }
    __syncthreads();
    __int128 sumD = 0;
    for (int w = 0; w < NWW; ++w)
        sumD += make_i128(s_hi[w], s_lo[w]);
    run = run0;
    const bool nodes = S.deposit == SIC_DEPOSIT_FIRST;  // E_j = (K_j + K_{j+1}) / 2
    for (int j = j0; j < j1; ++j) {
        const long long mj = S.mesh_last[j];
        const __int128 d = (__int128)nx * run - (__int128)j * qtot;
        const __int128 K = (__int128)nx * d - sumD;
        if (nodes) {
            const __int128 Kn = (__int128)nx * ((__int128)nx * (run + mj) - (__int128)(j + 1) * qtot) - sumD;
            S.E64[j] = i128_to_double(K + Kn) * (0.5 * S.E_scale);
        } else {
            S.E64[j] = i128_to_double(K) * S.E_scale;
        }
        S.rho64[j] = i128_to_double((__int128)nx * mj - qtot) * S.rho_scale;
        run += mj;
    }
}

__global__ void k_expand_horizontal(uint32_t *U, float *V, const uint32_t *ut, int32_t n, const float *vs,
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

}  // namespace

size_t step_smem_bytes(int nx_max, bool staged, bool per_q)
{
    // shared head, mesh lo/hi [nx], diff [nx + 2], E [nx + 1] (the epilogue
    // reuses mesh and E), then the warps' staging buffers
    // then per warp one staging buffer (two when staged) and a task list
    const size_t buf = staged ? (per_q ? WarpBuf<true, true>::bytes : WarpBuf<false, true>::bytes)
                              : (per_q ? WarpBuf<true, false>::bytes : WarpBuf<false, false>::bytes);
    return stage_offset(nx_max) + (size_t)NW * buf + (size_t)NW * WT * sizeof(unsigned short);
}

// Blocks of the step kernel that the SM's shared memory holds (registers cap
// them at SIC_K1_MIN_BLOCKS by the launch bounds).
static int blocks_by_smem(size_t smem)
{
    static int per_sm = 0;
    if (per_sm == 0) {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) == cudaSuccess && v > 0)
            per_sm = v;
        else
            per_sm = 228 * 1024;
    }
    const int n = (int)((size_t)per_sm / (smem + 1024));  // 1 KB reserved per block
    return std::min(n, SIC_K1_MIN_BLOCKS);
}

// Stage items through shared memory unless the staging buffers would cost an
// SM a block (large meshes): occupancy hides more latency than staging.
bool step_staged(int nx_max, bool per_q)
{
    return blocks_by_smem(step_smem_bytes(nx_max, true, per_q)) >= blocks_by_smem(step_smem_bytes(nx_max, false, per_q));
}

static long long g_launches = 0;
void count_launches(int64_t n) { __atomic_add_fetch(&g_launches, n, __ATOMIC_RELAXED); }
int64_t launches() { return __atomic_load_n(&g_launches, __ATOMIC_RELAXED); }

cudaError_t launch_step_kernel(const LaunchArgs &a, int grid, Mode mode, bool per_q, cudaStream_t s)
{
    switch (mode) {
    case MODE_STEP: {
        bool staged = step_staged(a.nx_max, per_q);
        if (a.staging == 1)
            staged = false;
        else if (a.staging == 2)
            staged = step_smem_bytes(a.nx_max, true, per_q) <= 227 * 1024;
        if (staged)
            return run_pd<true, true, true>(a, grid, per_q, s);
        return run_pd<true, true, false>(a, grid, per_q, s);
    }
    case MODE_DEPOSIT:
        return run_pd<false, true, false>(a, grid, per_q, s);
    default:
        return run_pd<true, false, false>(a, grid, per_q, s);
    }
}

int step_blocks_per_sm(int nx_max, Mode mode, bool per_q)
{
    switch (mode) {
    case MODE_STEP:
        if (step_staged(nx_max, per_q))
            return occ_pd<true, true, true>(nx_max, per_q);
        return occ_pd<true, true, false>(nx_max, per_q);
    case MODE_DEPOSIT:
        return occ_pd<false, true, false>(nx_max, per_q);
    default:
        return occ_pd<true, false, false>(nx_max, per_q);
    }
}

cudaError_t launch_field_out(const SimDev &sim, cudaStream_t s)
{
    k_field_out<<<1, 1024, 0, s>>>(sim);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_spectrum(const SimDev &sim, int field, cudaStream_t s)
{
    k_spectrum<<<sim.nx / 2 + 1, 256, 0, s>>>(sim, field);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_expand_horizontal(uint32_t *U, float *V, const uint32_t *u_template, int32_t n_template,
                                     const float *v_sheet, const int64_t *sheet_offset, int32_t n_sheets,
                                     cudaStream_t s)
{
    k_expand_horizontal<<<1216, 256, 0, s>>>(U, V, u_template, n_template, v_sheet, sheet_offset, n_sheets);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace sic

namespace sic {
namespace {

// ------------------------------------------------------------ moments ----
// Number density n and current density j of the box particles of the
// current state (Sec. 2.3, Eq. rho_sum and Eq. j_sum: zero order on cells;
// Sec. 2.4: first order on the nodes x_j = j dx, the velocity interpolated
// linearly along each particle).  One thread per work item, FP64, atomics
// into n and j (physical units: n = charge / length, j = n v).
__device__ void moments_one(double xa, double va, double xb, double vb, double q, double vbar, int weighting, int nx,
                            double dx, double *n, double *j)
{
    const double a = fmin(xa, xb), b = fmax(xa, xb);
    const long long ma = (long long)floor(a / dx), mb = (long long)floor(b / dx);
    auto cell = [&](long long m) {
        const long long r = m % nx;
        return (int)(r < 0 ? r + nx : r);
    };
    if (b == a) {
        if (weighting == 0) {
            atomicAdd(n + cell(ma), q / dx);
            atomicAdd(j + cell(ma), q * vbar / dx);
        } else {
            const double f = a / dx - (double)ma;
            atomicAdd(n + cell(ma), q * (1.0 - f) / dx);
            atomicAdd(n + cell(ma + 1), q * f / dx);
            atomicAdd(j + cell(ma), q * vbar * (1.0 - f) / dx);
            atomicAdd(j + cell(ma + 1), q * vbar * f / dx);
        }
        return;
    }
    const double len = xb - xa;
    const double dens = q / fabs(len);
    if (mb - ma > 64ll * nx)
        return;  // longer than 64 box lengths: left out (bounded work per thread)
    for (long long m = ma; m <= mb; ++m) {
        const double lo = fmax(a, (double)m * dx), hi = fmin(b, (double)(m + 1) * dx);
        if (!(hi > lo))
            continue;
        const int c0 = cell(m), c1 = cell(m + 1);
        if (weighting == 0) {
            atomicAdd(n + c0, dens * (hi - lo) / dx);
            atomicAdd(j + c0, dens * vbar * (hi - lo) / dx);
            continue;
        }
        // s = (x - m dx) / dx: node m weighs 1 - s, node m + 1 weighs s; the
        // velocity on the piece is p + r s
        const double s0 = lo / dx - (double)m, s1 = hi / dx - (double)m;
        const double i0 = (s1 - s0) * dx;
        const double i1 = 0.5 * (s1 * s1 - s0 * s0) * dx;
        const double i2 = (s1 * s1 * s1 - s0 * s0 * s0) * dx / 3.0;
        const double r = (vb - va) * dx / len;
        const double p = va + (vb - va) * ((double)m * dx - xa) / len;
        atomicAdd(n + c0, dens * (i0 - i1) / dx);
        atomicAdd(n + c1, dens * i1 / dx);
        atomicAdd(j + c0, dens * (p * (i0 - i1) + r * (i1 - i2)) / dx);
        atomicAdd(j + c1, dens * (p * i1 + r * i2) / dx);
    }
}

__global__ void k_moments(const SimDev S, int weighting, double L, double unit_q, double unit_v, double *n,
                          double *j)
{
    const int nx = S.nx;
    const double dx = L / nx;
    const int src = (int)S.sc->buf;
    const unsigned *U = S.U[src];
    const float *V = S.V[src];
    const double box = L * 0x1p-32, unit_p = L * 0x1p-30;  // box fraction, position unit
    for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < S.n_items; it += gridDim.x * blockDim.x) {
        const WorkItem W = S.items[it];
        const long long last = W.t0 + W.count - 1;
        for (long long t = W.t0; t <= last; ++t) {
            long long t1 = t + 1;
            unsigned shift = 0u;
            if (t == last) {
                if (W.halo < 0)
                    break;
                t1 = W.halo;
                shift = W.halo_shift;
            }
            // the particle's lower end inside the box, its far end one
            // segment (the 32-bit position difference) away
            const double xa = (double)(U[t] << SIC_POS_WIND_BITS) * box;
            const double xb = xa + (double)(int)(U[t1] + shift - U[t]) * unit_p;
            const double va = (double)V[t] * unit_v, vb = (double)V[t1] * unit_v;
            const double qa = S.Qh ? (double)S.Qh[t] : (double)W.qh, qb = S.Qh ? (double)S.Qh[t1] : (double)W.qh;
            const double vbar = (qa + qb) > 0 ? (qa * va + qb * vb) / (qa + qb) : 0.5 * (va + vb);
            // per-particle charges (refined sheets): the particle's own; else the
            // mean of its tracers' weights
            const double qs = S.seg_q ? qa : qa + qb;
            moments_one(xa, va, xb, vb, qs * unit_q, vbar, weighting, nx, dx, n, j);
        }
    }
}

}  // namespace

cudaError_t launch_moments(const SimDev &sim, int weighting, double box_length, double unit_q, double unit_v,
                           double *n, double *j, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(n, 0, sizeof(double) * (size_t)sim.nx, s);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(j, 0, sizeof(double) * (size_t)sim.nx, s);
    if (e != cudaSuccess)
        return e;
    const int grid = (int)std::min<long long>(4096, ((long long)sim.n_items + 255) / 256);
    k_moments<<<std::max(grid, 1), 256, 0, s>>>(sim, weighting, box_length, unit_q, unit_v, n, j);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace sic

namespace sic {
namespace {

// ---------------------------------------------------------- refinement ----
// Sec. 2.6: a particle longer than the refinement length (lfix, position
// units) gets a new tracer at its centre.  k_refine_count counts those
// particles per work item; k_refine_scatter writes every tracer, and after
// each split particle's first tracer the new one, into the new layout, with
// per-particle charges: each half of a split particle gets half its charge
// (the first floor(Q / 2), the second the rest).  One thread per work item.
__device__ __forceinline__ bool refine_seg(const WorkItem &W, long long t, const unsigned *U, long long &d,
                                           long long &t1)
{
    const long long last = W.t0 + W.count - 1;
    unsigned shift = 0u;
    t1 = t + 1;
    if (t == last) {
        if (W.halo < 0)
            return false;
        t1 = W.halo;
        shift = W.halo_shift;
    }
    d = (long long)(int)(U[t1] + shift - U[t]);
    return true;
}

__global__ void k_refine_count(const SimDev S, long long lfix, int32_t *splits)
{
    const unsigned *U = S.U[S.sc->buf & 1];
    for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < S.n_items; it += gridDim.x * blockDim.x) {
        const WorkItem W = S.items[it];
        int c = 0;
        for (long long t = W.t0; t < W.t0 + W.count; ++t) {
            long long d, t1;
            if (refine_seg(W, t, U, d, t1) && (d > lfix || -d > lfix))
                ++c;
        }
        splits[it] = c;
    }
}

__global__ void k_refine_scatter(const SimDev S, long long lfix, const int64_t *out_base, uint32_t *U2, float *V2,
                                 int32_t *Q2)
{
    const int b = (int)(S.sc->buf & 1);
    const unsigned *U = S.U[b];
    const float *V = S.V[b];
    for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < S.n_items; it += gridDim.x * blockDim.x) {
        const WorkItem W = S.items[it];
        long long out = out_base[it];
        for (long long t = W.t0; t < W.t0 + W.count; ++t) {
            long long d = 0, t1 = t;
            const bool seg = refine_seg(W, t, U, d, t1);
            // the particle's charge: its own (refined sheets), else the
            // mean of its tracers' weights (the sheet's, or per tracer)
            const int Q = !seg ? 0 : S.seg_q ? S.Qh[t] : S.Qh ? S.Qh[t] + S.Qh[t1] : 2 * W.qh;
            U2[out] = U[t];
            V2[out] = V[t];
            if (seg && (d > lfix || -d > lfix)) {
                Q2[out] = Q >> 1;
                ++out;
                U2[out] = U[t] + (unsigned)(int)(d >> 1);  // floor of half the segment
                V2[out] = 0.5f * (V[t] + V[t1]);
                Q2[out] = Q - (Q >> 1);
            } else {
                Q2[out] = Q;
            }
            ++out;
        }
    }
}

}  // namespace

cudaError_t launch_refine_count(const SimDev &sim, long long lfix, int32_t *splits, cudaStream_t s)
{
    const int grid = (int)std::max<long long>(1, std::min<long long>(4096, ((long long)sim.n_items + 255) / 256));
    k_refine_count<<<grid, 256, 0, s>>>(sim, lfix, splits);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_refine_scatter(const SimDev &sim, long long lfix, const int64_t *out_base, uint32_t *U2, float *V2,
                                  int32_t *Q2, cudaStream_t s)
{
    const int grid = (int)std::max<long long>(1, std::min<long long>(4096, ((long long)sim.n_items + 255) / 256));
    k_refine_scatter<<<grid, 256, 0, s>>>(sim, lfix, out_base, U2, V2, Q2);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace sic
