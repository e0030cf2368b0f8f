// core.cuh -- the Gray-code walk shared by every enumeration kernel.
//
// This header is compiled twice: by nvcc into the precompiled generic kernels
// (generic.cu) and, as source text, by NVRTC into every per-matrix kernel the
// code generator emits.  It therefore uses no standard headers.  (The host
// emulation tests also compile it, with a generated kernel, as host C++.)
//
// The walk (Algorithm 1, Nijenhuis-Wilf variant of Eq. 2).  The columns are in
// the plan's order, column n-1 is never flipped, and x is
//     x_i(g) = x0_i + sum_{j : bit j of Gray(g)} a_ij,
//     x0_i   = a_{i,n-1} - (1/2) sum_j a_ij            (FP64 path)
// or twice that (exact path, so that x stays integral).  Gray index g
// contributes (-1)^g prod_i x_i(g).
//
// Parallel layout (Sec. II-A, Theorem 1, Lemma 1).  The 2^(n-1) indices are
// cut into aligned chunks of 2^K; chunk q starts from x(q 2^K), built from the
// set bits of Gray(q 2^K) (all >= K-1).  The warp builds its 32 start vectors
// together: it visits every column set in any lane's code, and each lane adds
// that column with weight 0 or 1, so no lane waits for another's flips.
// Inside a chunk step l flips column j = ctz(l) with sign + iff bit j+1 of g
// is 0 (Theorem 1).  Because chunks are aligned powers of two, every lane of a
// warp flips the same column at the same step: only the sign of column K-1
// differs between lanes (the first case of Lemma 1), and that is an
// arithmetic sign, not a branch.  The second
// divergent case of Lemma 1 (l = 2^k) never arises because each chunk starts
// from its own start vector.  Chunks are grouped 32 per warp task; warps of a
// persistent grid take tasks from an atomic counter.
//
// Blocks.  A chunk is walked in blocks of 2^B steps.  The 2^B - 1 flips inside
// a block are columns 0..B-1 in the ruler order of SCBS(B) (Sec. IV); in the
// generated kernels they are fully unrolled with compile-time column, row set
// and sign (the generic kernels roll them into a loop).  The flip at a block
// boundary (column >= B) is chosen at run time, and it is uniform across the
// warp.
//
// Product chain.  Rows are grouped by the first ordered column that touches
// them: R_m.  A flip of column j changes only rows in R_0..R_j, so with
//     Q_m = prod of x over R_m, R_{m+1}, ..., R_{n-1}
// the product after the flip is Q_0, rebuilt from Q_{j+1} by |R_0|+...+|R_j|
// multiplications.  This generalises the reuse of globalProduct for
// register-only columns (Sec. V, Listings 4-5) to every level, and with the
// permanent ordering of Algorithm 3 the low levels hold few rows.  Every term
// is still the product of the same n numbers; only the association changes.
//
// Zero skip (Sec. VI-B's zero tracking, made warp-uniform; Sec. VI-E and
// Sec. VIII: repeated values make zero entries of x persist).  When Q_B is
// zero in every lane at a block boundary, all 2^B products of the block are
// zero: the block is replaced by its net effect on x (one flip of column
// B-1).  The skip then widens level by level: blocks h .. h+2^m-1, with h a
// multiple of 2^m, flip only columns below B+m, so Q_{B+m} is constant over
// them, and where it is zero in every lane the whole aligned span of 2^(B+m)
// steps is zero.  Over an aligned span of 2^(B+m) Gray indices every column
// below B+m-1 flips an even number of times and column B+m-1 once, at the
// middle index (sign by bit B+m of the span's start, Theorem 1), so the span's
// net effect on x is that one flip.  Levels B..B+m-1 go stale; the flip at
// the next block boundary is of a column >= B+m and rebuilds them.
#pragma once

#include "devmat.h"

typedef unsigned long long u64;
typedef unsigned int u32;
typedef long long i64;

#ifndef PERM_FULLMASK
#define PERM_FULLMASK 0xffffffffu
#endif

namespace pk {

__device__ __forceinline__ int ctz64(u64 v) { return __ffsll((long long)v) - 1; }

// OR of a 64-bit value over the 32 lanes of a (converged) warp.
__device__ __forceinline__ u64 warp_or64(u64 v) {
    const u32 lo = __reduce_or_sync(PERM_FULLMASK, (u32)v);
    const u32 hi = __reduce_or_sync(PERM_FULLMASK, (u32)(v >> 32));
    return ((u64)hi << 32) | lo;
}

// Nanoseconds from the GPU's global timer (0 when the walk code runs as
// host C++ in the emulation tests).
__device__ __forceinline__ u64 global_ns() {
    u64 t = 0;
#ifndef PERM_HOST_EMULATION
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
#endif
    return t;
}

// Device-side deadline.  The first warp to fetch a task stores "now +
// timeout" in *deadline_word; every warp compares the GPU clock with it
// before taking a task, and past it raises the abort flag and stops taking
// work.  Nothing ever waits on the flag or the word.
__device__ __forceinline__ bool past_deadline(u64 timeout_ns, u64 *deadline_word, unsigned int *abort_flag) {
    if (!timeout_ns) return false;
    const u64 now = global_ns();
    u64 d = *(volatile u64 *)deadline_word;
    if (!d) {
        atomicCAS(deadline_word, 0ull, now + timeout_ns);
        d = *(volatile u64 *)deadline_word;
    }
    if (now < d) return false;
    atomicExch(abort_flag, 1u);
    return true;
}

// ------------------------------------------------------------------ sum of |terms|
// Every FP64 (and double-double) walk also sums the absolute values of its
// terms, sum_g |prod_i x_i(g)|: the cancellation of the alternating sum
// (Sec. II) is that sum over |perm|, and it bounds the rounding error of the
// result.  It is accumulated on the FP32 pipe, so the FP64 pipe that bounds
// the walk does not see it: |t| 2^-shift is read from the high word of t with
// integer instructions (the exponent rebiased from 1023 to 127, the top 20
// fraction bits kept: relative error below 2^-20, always low), then added in
// FP32.  The per-matrix shift keeps the largest possible term near 2^120;
// values below 2^-126 after the shift count as zero, from 2^128 on they
// saturate.
__device__ __forceinline__ float abs_scaled_f32(double t, int shift) {
    int h = (__double2hiint(t) & 0x7fffffff) - (896 + shift) * (1 << 20);
    h = min(max(h, 0), 0x0fefffff);
    return __int_as_float(h << 3);
}

// ------------------------------------------------------------------ FP64 arithmetic

struct ArithF64 {
    typedef double X;   // an entry of x
    typedef double P;   // a (partial) product
    typedef double V;   // a matrix value as stored
    typedef double X0;  // a start value as stored
    // compensated sum (hi, lo) and the sum of |terms| (scaled by 2^-shift)
    struct Acc { double hi, lo, abs; };
    static constexpr bool kProdIsX = true;   // a product is itself a valid factor
    static __device__ __forceinline__ P one() { return 1.0; }
    static __device__ __forceinline__ P mul(P q, X x) { return q * x; }
    static __device__ __forceinline__ P diff(P a, P b) { return a - b; }
    static __device__ __forceinline__ bool is_zero(P q) { return q == 0.0; }
    template <int S> static __device__ __forceinline__ X upd(X x, V v) { return S > 0 ? x + v : x - v; }
    // x + s v for s = +1, -1 or 0 (the start vector adds a column with weight 0
    // or 1): the sign goes into v's sign bit with an integer instruction, so
    // the FP64 pipe sees one addition (converting s to a double and fusing
    // s * v + x cost the pipe a conversion as well: 11 % of the generic walk)
    static __device__ __forceinline__ X upd_rt(X x, V v, int s) {
        const double sv = __hiloint2double(__double2hiint(v) ^ (s < 0 ? (int)0x80000000 : 0), __double2loint(v));
        return s == 0 ? x : x + sv;
    }
    static __device__ __forceinline__ X load_x0(const volatile void *base, int i) {
        return ((const volatile double *)base)[i];
    }
    // block accumulator: a plain double over 2^B terms, and their |terms| in FP32
    struct Blk { double s; float a; };
    static __device__ __forceinline__ Blk blk_zero() { Blk b; b.s = 0.0; b.a = 0.f; return b; }
    template <int S> static __device__ __forceinline__ void blk_add(Blk &b, P p) { if (S > 0) b.s += p; else b.s -= p; }
    // |t| of one term, and an already scaled FP32 contribution
    static __device__ __forceinline__ void blk_abs(Blk &b, P t, int shift) { b.a += abs_scaled_f32(t, shift); }
    static __device__ __forceinline__ void blk_abs_f(Blk &b, float f) { b.a += f; }
    static __device__ __forceinline__ void blk_accumulate(Blk &a, Blk b) { a.s += b.s; a.a += b.a; }
    static __device__ __forceinline__ Acc acc_zero() { Acc a; a.hi = 0.0; a.lo = 0.0; a.abs = 0.0; return a; }
    // TwoSum (Knuth): a.hi + b = s + e exactly
    static __device__ __forceinline__ void acc_merge(Acc &a, Blk b) {
        double s = a.hi + b.s;
        double bb = s - a.hi;
        double e = (a.hi - (s - bb)) + (b.s - bb);
        a.hi = s;
        a.lo += e;
        a.abs += (double)b.a;
    }
    static __device__ __forceinline__ Acc acc_add(Acc a, Acc b) {
        double s = a.hi + b.hi;
        double bb = s - a.hi;
        double e = (a.hi - (s - bb)) + (b.hi - bb);
        e += a.lo + b.lo;
        Acc r;
        r.hi = s + e;
        r.lo = e - (r.hi - s);
        r.abs = a.abs + b.abs;
        return r;
    }
    static __device__ __forceinline__ Acc shfl_down(Acc a, int d) {
        Acc r;
        r.hi = __shfl_down_sync(PERM_FULLMASK, a.hi, d);
        r.lo = __shfl_down_sync(PERM_FULLMASK, a.lo, d);
        r.abs = __shfl_down_sync(PERM_FULLMASK, a.abs, d);
        return r;
    }
    static constexpr int ACC_WORDS = 3;   // stored as three doubles
    static __device__ __forceinline__ void acc_store(u64 *dst, Acc a) {
        dst[0] = (u64)__double_as_longlong(a.hi);
        dst[1] = (u64)__double_as_longlong(a.lo);
        dst[2] = (u64)__double_as_longlong(a.abs);
    }
    static __device__ __forceinline__ Acc acc_load(const u64 *src) {
        Acc a;
        a.hi = __longlong_as_double((long long)src[0]);
        a.lo = __longlong_as_double((long long)src[1]);
        a.abs = __longlong_as_double((long long)src[2]);
        return a;
    }
};

// ------------------------------------------------------------------ double-double arithmetic
// For ill-conditioned FP64 inputs (sum|terms| / |perm| large): every x_i,
// product and sum is an unevaluated pair of doubles h + l (about 106 bits).
// x updates are exact TwoSum additions (Knuth), products are FMA-based exact
// products of the high parts (Dekker's two-product, done with one fused
// multiply-add) plus the cross terms, so a term carries a relative error of a
// few 2^-104 instead of n 2^-53.  Same walk, same terms; only the precision of
// each operation changes.  The results use the FP64 accumulator and reduction.

struct DD { double h, l; };

struct ArithDD {
    typedef DD X;
    typedef DD P;
    typedef double V;
    typedef DD X0;
    typedef ArithF64::Acc Acc;
    static constexpr bool kProdIsX = true;
    static __device__ __forceinline__ DD mk(double h, double l) { DD r; r.h = h; r.l = l; return r; }
    static __device__ __forceinline__ P one() { return mk(1.0, 0.0); }
    // (q.h + q.l)(x.h + x.l) ~ p + e: p = q.h x.h rounded, e = its exact error
    // (one FMA) plus the cross terms; q.l x.l (below 2^-104 relative) dropped
    static __device__ __forceinline__ P mul(P q, X x) {
        const double p = q.h * x.h;
        double e = fma(q.h, x.h, -p);
        e = fma(q.h, x.l, e);
        e = fma(q.l, x.h, e);
        return mk(p, e);
    }
    // (a.h + a.l) + b, renormalised so that |l| <= ulp(h)/2
    static __device__ __forceinline__ DD add_d(DD a, double b) {
        const double s = a.h + b;
        const double bb = s - a.h;
        const double e = (a.h - (s - bb)) + (b - bb);
        const double l = a.l + e;
        const double h = s + l;
        return mk(h, l - (h - s));
    }
    static __device__ __forceinline__ DD add_dd(DD a, DD b) {
        const double s = a.h + b.h;
        const double bb = s - a.h;
        double e = (a.h - (s - bb)) + (b.h - bb);
        e += a.l + b.l;
        const double h = s + e;
        return mk(h, e - (h - s));
    }
    static __device__ __forceinline__ double neg_if(double v, int s) {
        return s < 0 ? __hiloint2double(__double2hiint(v) ^ (int)0x80000000, __double2loint(v)) : v;
    }
    static __device__ __forceinline__ P diff(P a, P b) { return add_dd(a, mk(-b.h, -b.l)); }
    static __device__ __forceinline__ bool is_zero(P q) { return q.h == 0.0 && q.l == 0.0; }
    template <int S> static __device__ __forceinline__ X upd(X x, V v) { return add_d(x, S > 0 ? v : -v); }
    // s is +1, -1 or 0 (the start vector adds a column with weight 0 or 1)
    static __device__ __forceinline__ X upd_rt(X x, V v, int s) { return s == 0 ? x : add_d(x, neg_if(v, s)); }
    static __device__ __forceinline__ X load_x0(const volatile void *base, int i) {
        const volatile double *d = (const volatile double *)base;
        return mk(d[2 * i], d[2 * i + 1]);
    }
    struct Blk { DD s; float a; };
    static __device__ __forceinline__ Blk blk_zero() { Blk b; b.s = mk(0.0, 0.0); b.a = 0.f; return b; }
    template <int S> static __device__ __forceinline__ void blk_add(Blk &b, P p) {
        b.s = add_dd(b.s, S > 0 ? p : mk(-p.h, -p.l));
    }
    static __device__ __forceinline__ void blk_abs(Blk &b, P t, int shift) { b.a += abs_scaled_f32(t.h, shift); }
    static __device__ __forceinline__ void blk_abs_f(Blk &b, float f) { b.a += f; }
    static __device__ __forceinline__ void blk_accumulate(Blk &a, Blk b) { a.s = add_dd(a.s, b.s); a.a += b.a; }
    static __device__ __forceinline__ Acc acc_zero() { return ArithF64::acc_zero(); }
    static __device__ __forceinline__ void acc_merge(Acc &a, Blk b) {
        double s = a.hi + b.s.h;
        double bb = s - a.hi;
        double e = (a.hi - (s - bb)) + (b.s.h - bb);
        a.hi = s;
        a.lo += e + b.s.l;
        a.abs += (double)b.a;
    }
    static __device__ __forceinline__ Acc acc_add(Acc a, Acc b) { return ArithF64::acc_add(a, b); }
    static __device__ __forceinline__ Acc shfl_down(Acc a, int d) { return ArithF64::shfl_down(a, d); }
    static constexpr int ACC_WORDS = ArithF64::ACC_WORDS;
    static __device__ __forceinline__ void acc_store(u64 *dst, Acc a) { ArithF64::acc_store(dst, a); }
    static __device__ __forceinline__ Acc acc_load(const u64 *src) { return ArithF64::acc_load(src); }
};

// ------------------------------------------------------------------ exact arithmetic
// Products live in Z / 2^(32 L): L little-endian 32-bit limbs.  x entries are
// signed 32-bit (twice the Nijenhuis-Wilf row sums).  Wrapping arithmetic is a
// ring homomorphism, so the final sum is exact modulo 2^(32 L).

template <int L> struct Ring { u32 w[L]; };

template <int L>
__device__ __forceinline__ Ring<L> ring_mul(const Ring<L> &q, int x) {
    // q * (x mod 2^32), then subtract q * 2^32 when x < 0 (two's complement).
    Ring<L> r;
    u32 m = (u32)x;
    u64 c = 0;
#pragma unroll
    for (int i = 0; i < L; ++i) {
        u64 t = (u64)q.w[i] * m + c;
        r.w[i] = (u32)t;
        c = t >> 32;
    }
    if (x < 0) {
        u32 borrow = 0;
#pragma unroll
        for (int i = 1; i < L; ++i) {
            u64 t = (u64)r.w[i] - (u64)q.w[i - 1] - (u64)borrow;
            r.w[i] = (u32)t;
            borrow = (u32)(t >> 63);
        }
    }
    return r;
}

template <>
__device__ __forceinline__ Ring<2> ring_mul<2>(const Ring<2> &q, int x) {
    u64 v = ((u64)q.w[1] << 32) | q.w[0];
    v *= (u64)(i64)x;
    Ring<2> r;
    r.w[0] = (u32)v;
    r.w[1] = (u32)(v >> 32);
    return r;
}

template <int L>
__device__ __forceinline__ void ring_add(Ring<L> &a, const Ring<L> &b) {
    u32 c = 0;
#pragma unroll
    for (int i = 0; i < L; ++i) {
        u64 t = (u64)a.w[i] + b.w[i] + c;
        a.w[i] = (u32)t;
        c = (u32)(t >> 32);
    }
}

template <int L>
__device__ __forceinline__ void ring_sub(Ring<L> &a, const Ring<L> &b) {
    u32 br = 0;
#pragma unroll
    for (int i = 0; i < L; ++i) {
        u64 t = (u64)a.w[i] - (u64)b.w[i] - (u64)br;
        a.w[i] = (u32)t;
        br = (u32)(t >> 63);
    }
}

template <>
__device__ __forceinline__ void ring_add<2>(Ring<2> &a, const Ring<2> &b) {
    u64 v = (((u64)a.w[1] << 32) | a.w[0]) + (((u64)b.w[1] << 32) | b.w[0]);
    a.w[0] = (u32)v;
    a.w[1] = (u32)(v >> 32);
}

template <>
__device__ __forceinline__ void ring_sub<2>(Ring<2> &a, const Ring<2> &b) {
    u64 v = (((u64)a.w[1] << 32) | a.w[0]) - (((u64)b.w[1] << 32) | b.w[0]);
    a.w[0] = (u32)v;
    a.w[1] = (u32)(v >> 32);
}

// Exact arithmetic in Z / 2^(32 NL): NL 32-bit limbs, stored and reduced as
// ceil(NL/2) 64-bit words (an odd limb count leaves the top half-word of the
// last word zero; sums of stored words stay right modulo 2^(32 NL)).
template <int NL>
struct ArithExact {
    static constexpr int L = NL;
    static constexpr int W = (NL + 1) / 2;
    typedef int X;
    typedef Ring<L> P;
    typedef int V;
    typedef int X0;
    typedef Ring<L> Acc;
    typedef Ring<L> Blk;
    static __device__ __forceinline__ X load_x0(const volatile void *base, int i) { return ((const volatile int *)base)[i]; }
    static __device__ __forceinline__ void blk_abs(Blk &, const P &, int) {}
    static __device__ __forceinline__ void blk_abs_f(Blk &, float) {}
    static __device__ __forceinline__ P one() {
        P r;
#pragma unroll
        for (int i = 0; i < L; ++i) r.w[i] = 0;
        r.w[0] = 1;
        return r;
    }
    static constexpr bool kProdIsX = false;
    static __device__ __forceinline__ P mul(const P &q, X x) { return ring_mul<L>(q, x); }
    static __device__ __forceinline__ P diff(P a, const P &b) { ring_sub<L>(a, b); return a; }
    static __device__ __forceinline__ bool is_zero(const P &q) {
        u32 o = 0;
#pragma unroll
        for (int i = 0; i < L; ++i) o |= q.w[i];
        return o == 0;
    }
    template <int S> static __device__ __forceinline__ X upd(X x, V v) { return S > 0 ? x + v : x - v; }
    static __device__ __forceinline__ X upd_rt(X x, V v, int s) { return x + s * v; }
    static __device__ __forceinline__ Blk blk_zero() {
        Blk r;
#pragma unroll
        for (int i = 0; i < L; ++i) r.w[i] = 0;
        return r;
    }
    template <int S> static __device__ __forceinline__ void blk_add(Blk &b, const P &p) {
        if (S > 0) ring_add<L>(b, p); else ring_sub<L>(b, p);
    }
    static __device__ __forceinline__ void blk_accumulate(Blk &a, const Blk &b) { ring_add<L>(a, b); }
    static __device__ __forceinline__ Acc acc_zero() { return blk_zero(); }
    static __device__ __forceinline__ void acc_merge(Acc &a, const Blk &b) { ring_add<L>(a, b); }
    static __device__ __forceinline__ Acc acc_add(Acc a, const Acc &b) { ring_add<L>(a, b); return a; }
    static __device__ __forceinline__ Acc shfl_down(const Acc &a, int d) {
        Acc r;
#pragma unroll
        for (int i = 0; i < L; ++i) r.w[i] = __shfl_down_sync(PERM_FULLMASK, a.w[i], d);
        return r;
    }
    static constexpr int ACC_WORDS = W;
    static __device__ __forceinline__ void acc_store(u64 *dst, const Acc &a) {
#pragma unroll
        for (int i = 0; i < W; ++i) {
            const u64 hi = (2 * i + 1 < L) ? (u64)a.w[(2 * i + 1) % L] : 0ull;
            dst[i] = (hi << 32) | a.w[2 * i];
        }
    }
    static __device__ __forceinline__ Acc acc_load(const u64 *src) {
        Acc a;
#pragma unroll
        for (int i = 0; i < W; ++i) {
            a.w[2 * i] = (u32)src[i];
            if (2 * i + 1 < L) a.w[(2 * i + 1) % L] = (u32)(src[i] >> 32);
        }
        return a;
    }
};

// Adds |t| of one term to the block's sum of |terms|, if the policy keeps it.
template <class Pol, class A>
__device__ __forceinline__ void term_abs(const Pol &pol, typename A::Blk &blk, const typename A::P &t) {
    if constexpr (Pol::kAbs) A::blk_abs(blk, t, pol.abs_shift);
}

// ------------------------------------------------------------------ the unrolled block
// Step l (1 <= l < 2^B) of a block flips column J = ctz(l).  Its sign is bit
// J+1 of l for J < B-1; for J = B-1 it is bit B of the block start, passed in
// as s_mid.  The term's sign (-1)^g equals (-1)^l because every block starts
// at an even index.

template <int Lstep> struct Ctz { static constexpr int v = (Lstep & 1) ? 0 : 1 + Ctz<(Lstep >> 1)>::v; };
template <> struct Ctz<0> { static constexpr int v = 0; };

// Rebuilds chain levels M, M-1, ..., 1 (Q[m] = Q[m+1] * prod over R_m).
template <class Pol, class A, int Bv, int M>
struct LevelsDown {
    static __device__ __forceinline__ void run(Pol &pol, typename A::X (&x)[Pol::NX], typename A::P (&Q)[Bv + 1]) {
        if constexpr (M >= 1) {
            Q[M] = pol.template grp<M>(x, Q[M + 1]);
            LevelsDown<Pol, A, Bv, M - 1>::run(pol, x, Q);
        }
    }
};

template <class Pol, class A, int Bv, int Lstep>
struct BlockSteps {
    static __device__ __forceinline__ void run(Pol &pol, typename A::X (&x)[Pol::NX], typename A::P (&Q)[Bv + 1],
                                               typename A::Blk &blk, int s_mid) {
        if constexpr (Lstep < (1 << Bv)) {
            constexpr int J = Ctz<Lstep>::v;
            if constexpr (J == Bv - 1) {
                pol.template flip_rt<J>(x, s_mid);
            } else {
                constexpr int S = ((Lstep >> (J + 1)) & 1) ? -1 : 1;
                pol.template flip<J, S>(x);
            }
            LevelsDown<Pol, A, Bv, J>::run(pol, x, Q);
            typename A::P p = pol.template grp<0>(x, Q[1]);
            A::template blk_add<(Lstep & 1) ? -1 : 1>(blk, p);
            term_abs<Pol, A>(pol, blk, p);
            BlockSteps<Pol, A, Bv, Lstep + 1>::run(pol, x, Q, blk, s_mid);
        }
    }
};

// Paired form (policies with kPaired): an even step l (flip of column
// J = ctz(l) >= 1, then levels J..1 rebuilt) and the odd step l+1 (flip of
// column 0, sign bit 1 of l+1) differ only in the rows of R_0, which are
// exactly column 0's rows, so their two terms combine into
//   (-1)^l (P(l) - P(l+1)) = Q_1 (prod_{R_0} x - prod_{R_0} (x + s a_0)),
// formed once by the policy's pair<s>() (which also applies the column-0
// flip, and returns |P(l)| + |P(l+1)|, scaled, in FP32 through its last
// argument).  Same terms, about 1.5 fewer multiply/add operations per step.
template <class Pol, class A, int Bv, int Lstep>
struct PairSteps {
    static __device__ __forceinline__ void run(Pol &pol, typename A::X (&x)[Pol::NX], typename A::P (&Q)[Bv + 1],
                                               typename A::Blk &blk, int s_mid) {
        if constexpr (Lstep < (1 << Bv)) {
            constexpr int J = Ctz<Lstep>::v;     // >= 1: Lstep is even
            if constexpr (J == Bv - 1) {
                pol.template flip_rt<J>(x, s_mid);
            } else {
                constexpr int S = ((Lstep >> (J + 1)) & 1) ? -1 : 1;
                pol.template flip<J, S>(x);
            }
            LevelsDown<Pol, A, Bv, J>::run(pol, x, Q);
            constexpr int S0 = (((Lstep + 1) >> 1) & 1) ? -1 : 1;
            float fa;
            A::template blk_add<1>(blk, pol.template pair<S0>(x, Q[1], fa));
            if constexpr (Pol::kAbs) A::blk_abs_f(blk, fa);
            PairSteps<Pol, A, Bv, Lstep + 2>::run(pol, x, Q, blk, s_mid);
        }
    }
};

// ------------------------------------------------------------------ zero spans
// At block h of a chunk of 2^K steps whose block products are all zero (every
// lane), the largest m such that the aligned span of blocks h .. h+2^m-1 is
// all zero too: m <= ctz(h) (the whole chunk at h = 0), and Q_{B+m} zero in
// every lane.  Zero levels are nested (Q_{B+m} is Q_{B+m+1} times more rows),
// so the search climbs until a level is nonzero in some lane.
template <class Pol, int Bv>
__device__ __forceinline__ int zero_span(const Pol &pol, u64 h, int K) {
    if constexpr (!Pol::kZeroSpans) return 0;   // a kernel built without the wider skip
    const int t = h ? ctz64(h) : K - Bv;
    int m = 0;
    while (m < t && __all_sync(PERM_FULLMASK, pol.level_zero(Bv + m + 1))) ++m;
    return m;
}

// ------------------------------------------------------------------ two-state chains
// Policies with kDual never apply column 0 to x.  A step's product is
//     prod_i x_i = (column 0 off) ? A_1 : B_1,
// where, over the rows of column 0 (group 0), A_m takes x_i and B_m takes
// x_i + a_i0.  Group 0's rows are split by the next column that touches them
// (S_m), and level m of both chains holds group m and S_m:
//     A_m = A_{m+1} prod_{R_m} x prod_{S_m} x,
//     B_m = B_{m+1} prod_{R_m} x prod_{S_m} (x + a_0),
// so a flip of column j >= 1 rebuilds levels j..1 of both, and column 0's
// steps cost nothing.  Steps 2p and 2p+1 of a block differ only in column 0
// (off, then on, for even p; on, then off, for odd p), so the pair adds
// (-1)^p (A_1 - B_1).  The flip before pair p is column 1 + ctz(p), sign bit
// 1 + ctz(p) of p.  Every term is still the product of the same n numbers.
template <class Pol, class A, int Bv>
__device__ __forceinline__ void dual_block(Pol &pol, typename A::X (&x)[Pol::NX], typename A::P (&QA)[Bv + 1],
                                           typename A::P (&QB)[Bv + 1], typename A::Blk &blk, int s_mid) {
    static_assert(Bv >= 3, "the two-state block walks groups of two pairs");
#pragma unroll 1
    for (int p2 = 0; p2 < (1 << (Bv - 2)); ++p2) {
        if (p2 != 0) {
            const int p = p2 << 1;
            const int j = __ffs(p);   // 1 + ctz(p), >= 2
            const int s = (j == Bv - 1) ? s_mid : (((p >> j) & 1) ? -1 : 1);
            pol.flip_dyn(j, x, s);
#pragma unroll
            for (int M = Bv - 1; M >= 1; --M)
                if (M <= j) pol.level2(M, x, QA[M + 1], QB[M + 1], QA[M], QB[M]);
        }
        A::template blk_add<1>(blk, A::diff(QA[1], QB[1]));
        term_abs<Pol, A>(pol, blk, QA[1]);
        term_abs<Pol, A>(pol, blk, QB[1]);
        pol.flip_dyn(1, x, (p2 & 1) ? -1 : 1);
        pol.level2(1, x, QA[2], QB[2], QA[1], QB[1]);
        A::template blk_add<-1>(blk, A::diff(QA[1], QB[1]));
        term_abs<Pol, A>(pol, blk, QA[1]);
        term_abs<Pol, A>(pol, blk, QB[1]);
    }
}

// The same block unrolled (generated kernels): pair P's flip has a
// compile-time column and sign, and level2c<M> compile-time rows.
template <class Pol, class A, int Bv, int M>
struct LevelsDown2 {
    static __device__ __forceinline__ void run(Pol &pol, typename A::X (&x)[Pol::NX], typename A::P (&QA)[Bv + 1],
                                               typename A::P (&QB)[Bv + 1]) {
        if constexpr (M >= 1) {
            pol.template level2c<M>(x, QA[M + 1], QB[M + 1], QA[M], QB[M]);
            LevelsDown2<Pol, A, Bv, M - 1>::run(pol, x, QA, QB);
        }
    }
};

template <class Pol, class A, int Bv, int Pp>
struct DualSteps {
    static __device__ __forceinline__ void run(Pol &pol, typename A::X (&x)[Pol::NX], typename A::P (&QA)[Bv + 1],
                                               typename A::P (&QB)[Bv + 1], typename A::Blk &blk, int s_mid) {
        if constexpr (Pp < (1 << (Bv - 1))) {
            if constexpr (Pp > 0) {
                constexpr int J = 1 + Ctz<Pp>::v;
                if constexpr (J == Bv - 1) {
                    pol.template flip_rt<J>(x, s_mid);
                } else {
                    constexpr int S = ((Pp >> J) & 1) ? -1 : 1;
                    pol.template flip<J, S>(x);
                }
                LevelsDown2<Pol, A, Bv, J>::run(pol, x, QA, QB);
            }
            A::template blk_add<(Pp & 1) ? -1 : 1>(blk, A::diff(QA[1], QB[1]));
            term_abs<Pol, A>(pol, blk, QA[1]);
            term_abs<Pol, A>(pol, blk, QB[1]);
            DualSteps<Pol, A, Bv, Pp + 1>::run(pol, x, QA, QB, blk, s_mid);
        }
    }
};

template <class Pol, class A, int Bv>
__device__ __forceinline__ typename A::Acc walk_chunk_dual(Pol &pol, u64 q, int K, int zero_skip, u64 &skipped) {
    typedef typename A::X X;
    typedef typename A::P P;
    X x[Pol::NX];
    const u64 g0 = q << K;
    pol.init_x(x, g0 ^ (g0 >> 1));   // bit 0 of the code is 0: column 0 off
    P QA, QB;
    pol.chain_init2(x, QA, QB);
    typename A::Acc acc = A::acc_zero();
    typename A::Blk mid = A::blk_zero();
    const u64 nblocks = 1ull << (K - Bv);
    u64 h = 0;
    int fj = -1, fs = 1;   // the run-time flip due before block h (see walk_chunk_single)
    bool net = false;
    for (;;) {
        if (fj >= 0) {
            pol.flip_dyn(fj, x, fs);
            if (net) {
                net = false;
                if (h >= nblocks) break;
                fj = Bv + ctz64(h);
                fs = (((g0 + (h << Bv)) >> (fj + 1)) & 1ull) ? -1 : 1;
                continue;
            }
            pol.chain_hi2(fj, x, QA, QB);
        }
        if (h != 0 && (h & 7) == 0) {
            A::acc_merge(acc, mid);
            mid = A::blk_zero();
        }
        const u64 gb = g0 + (h << Bv);
        const int s_mid = ((gb >> Bv) & 1ull) ? -1 : 1;
        // the vote is also the warp's reconvergence point (see walk_chunk_single)
        const bool all_zero = __all_sync(PERM_FULLMASK, A::is_zero(QA) && A::is_zero(QB));
        if (zero_skip && all_zero) {
            const int m = zero_span<Pol, Bv>(pol, h, K);
            skipped += 1ull << m;
            if (m == 0) {
                pol.template flip_rt<Bv - 1>(x, s_mid);
                if (++h >= nblocks) break;
                fj = Bv + ctz64(h);
                fs = (((g0 + (h << Bv)) >> (fj + 1)) & 1ull) ? -1 : 1;
            } else {
                fj = Bv + m - 1;
                fs = ((gb >> (Bv + m)) & 1ull) ? -1 : 1;
                net = true;
                h += 1ull << m;
            }
            continue;
        }
        P LA[Bv + 1], LB[Bv + 1];
        LA[Bv] = QA;
        LB[Bv] = QB;
#pragma unroll
        for (int M = Bv - 1; M >= 1; --M) pol.level2(M, x, LA[M + 1], LB[M + 1], LA[M], LB[M]);
        typename A::Blk blk = A::blk_zero();
        if constexpr (Pol::kUnrolledDual) DualSteps<Pol, A, Bv, 0>::run(pol, x, LA, LB, blk, s_mid);
        else dual_block<Pol, A, Bv>(pol, x, LA, LB, blk, s_mid);
        A::blk_accumulate(mid, blk);
        if (++h >= nblocks) break;
        fj = Bv + ctz64(h);
        fs = (((g0 + (h << Bv)) >> (fj + 1)) & 1ull) ? -1 : 1;
    }
    A::acc_merge(acc, mid);
    return acc;
}

// ------------------------------------------------------------------ one chunk
// Walks Gray indices [q 2^K, (q+1) 2^K) and returns sum (-1)^g prod_i x_i(g).

template <class Pol, class A, int Bv>
__device__ __forceinline__ typename A::Acc walk_chunk_single(Pol &pol, u64 q, int K, int zero_skip, u64 &skipped) {
    typedef typename A::X X;
    typedef typename A::P P;
    X x[Pol::NX];
    const u64 g0 = q << K;
    pol.init_x(x, g0 ^ (g0 >> 1));
    P QB = pol.chain_init(x);
    typename A::Acc acc = A::acc_zero();
    // block sums go into a plain mid-level sum, merged into the compensated
    // accumulator every 8 blocks (and at the end of the chunk)
    typename A::Blk mid = A::blk_zero();
    const u64 nblocks = 1ull << (K - Bv);
    u64 h = 0;
    // The run-time flips of x (a block boundary's, a zero span's net flip)
    // share one call site: in a generated kernel each site inlines the
    // literal updates of every column.
    int fj = -1, fs = 1;   // the flip due before block h (none at the chunk start)
    bool net = false;      // it is a zero span's net flip, and block h's own flip follows
    for (;;) {
        if (fj >= 0) {
            pol.flip_dyn(fj, x, fs);
            if (net) {
                net = false;
                if (h >= nblocks) break;
                fj = Bv + ctz64(h);
                fs = (((g0 + (h << Bv)) >> (fj + 1)) & 1ull) ? -1 : 1;
                continue;
            }
            QB = pol.chain_hi(fj, x);
        }
        if (h != 0 && (h & 7) == 0) {
            A::acc_merge(acc, mid);
            mid = A::blk_zero();
        }
        const u64 gb = g0 + (h << Bv);
        const int s_mid = ((gb >> Bv) & 1ull) ? -1 : 1;
        // The vote runs every block, skip or not: it is also the point where
        // the warp reconverges after the data-driven loops of a flip.
        const bool all_zero = __all_sync(PERM_FULLMASK, A::is_zero(QB));
        if (zero_skip && all_zero) {
            // every product of this block (and of the widest zero span that
            // starts here) is zero; apply the span's net flip
            const int m = zero_span<Pol, Bv>(pol, h, K);
            skipped += 1ull << m;
            if (m == 0) {
                pol.template flip_rt<Bv - 1>(x, s_mid);
                if (++h >= nblocks) break;
                fj = Bv + ctz64(h);
                fs = (((g0 + (h << Bv)) >> (fj + 1)) & 1ull) ? -1 : 1;
            } else {
                fj = Bv + m - 1;
                fs = ((gb >> (Bv + m)) & 1ull) ? -1 : 1;
                net = true;
                h += 1ull << m;
            }
            continue;
        }
        P Q[Bv + 1];
        Q[Bv] = QB;
        LevelsDown<Pol, A, Bv, Bv - 1>::run(pol, x, Q);
        typename A::Blk blk = A::blk_zero();
        if constexpr (Pol::kPaired) {
            // steps 0 and 1 (column 0, sign +: bit 1 of 1 is 0), then pairs (2,3), (4,5), ...
            float fa;
            A::template blk_add<1>(blk, pol.template pair<1>(x, Q[1], fa));
            if constexpr (Pol::kAbs) A::blk_abs_f(blk, fa);
            PairSteps<Pol, A, Bv, 2>::run(pol, x, Q, blk, s_mid);
        } else {
            const typename A::P p0 = pol.template grp<0>(x, Q[1]);
            A::template blk_add<1>(blk, p0);
            term_abs<Pol, A>(pol, blk, p0);
            BlockSteps<Pol, A, Bv, 1>::run(pol, x, Q, blk, s_mid);
        }
        A::blk_accumulate(mid, blk);
        if (++h >= nblocks) break;
        fj = Bv + ctz64(h);
        fs = (((g0 + (h << Bv)) >> (fj + 1)) & 1ull) ? -1 : 1;
    }
    A::acc_merge(acc, mid);
    return acc;
}

template <class Pol, class A, int Bv>
__device__ __forceinline__ typename A::Acc walk_chunk(Pol &pol, u64 q, int K, int zero_skip, u64 &skipped) {
    if constexpr (Pol::kDual) return walk_chunk_dual<Pol, A, Bv>(pol, q, K, zero_skip, skipped);
    else return walk_chunk_single<Pol, A, Bv>(pol, q, K, zero_skip, skipped);
}

// ------------------------------------------------------------------ persistent warp loop

template <class Pol, class A, int Bv>
__device__ __forceinline__ void walk_tasks(Pol &pol, const WalkArgs &wa) {
    const int lane = threadIdx.x & 31;
    u64 skipped = 0;
    for (;;) {
        u64 task = 0;
        if (lane == 0) task = past_deadline(wa.timeout_ns, wa.deadline_word, wa.abort_flag) ? ~0ull : atomicAdd(wa.task_counter, 1ull);
        task = __shfl_sync(PERM_FULLMASK, task, 0);
        if (task >= wa.ntasks) break;
        u64 q = wa.chunk_lo + task * 32ull + (u64)lane;
        const bool live = q < wa.chunk_hi;
        if (!live) q = wa.chunk_hi - 1;     // idle lanes shadow a real chunk to stay in step
        typename A::Acc acc = walk_chunk<Pol, A, Bv>(pol, q, wa.K, wa.zero_skip, skipped);
        if (!live) acc = A::acc_zero();
#pragma unroll
        for (int d = 16; d >= 1; d >>= 1) acc = A::acc_add(acc, A::shfl_down(acc, d));
        if (lane == 0) A::acc_store(wa.task_out + task * (u64)A::ACC_WORDS, acc);
    }
    // the warp's skipped blocks (a skip is warp-wide: one count per warp block)
    if (wa.skip_counter && lane == 0 && skipped) atomicAdd(wa.skip_counter, skipped);
}

// ------------------------------------------------------------------ final reduction
// One block sums the task results in a fixed order (deterministic).

template <class A>
__device__ __forceinline__ void reduce_tasks(const u64 *task_out, u64 ntasks, u64 *result) {
    __shared__ u64 sh[32 * 6];
    typename A::Acc acc = A::acc_zero();
    for (u64 t = threadIdx.x; t < ntasks; t += blockDim.x)
        acc = A::acc_add(acc, A::acc_load(task_out + t * (u64)A::ACC_WORDS));
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) acc = A::acc_add(acc, A::shfl_down(acc, d));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) A::acc_store(sh + warp * A::ACC_WORDS, acc);
    __syncthreads();
    if (warp == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        acc = lane < nw ? A::acc_load(sh + lane * A::ACC_WORDS) : A::acc_zero();
#pragma unroll
        for (int d = 16; d >= 1; d >>= 1) acc = A::acc_add(acc, A::shfl_down(acc, d));
        if (lane == 0) A::acc_store(result, acc);
    }
}

}  // namespace pk
