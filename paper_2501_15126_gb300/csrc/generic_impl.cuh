// generic_impl.cuh -- precompiled enumeration kernels (no per-matrix compilation).
//
// The Gray-code walk of core.cuh with a matrix policy that reads the ordered
// matrix from a compact image in shared memory.  x stays in registers (the
// register-allocation condition of Sec. III-A) without knowing the sparsity
// pattern at compile time: every access to x goes through a switch whose
// cases name x[k] with a compile-time k.  FP64 walks use the two-state chains
// of core.cuh (walk_chunk_dual); exact walks (and FP64 at 48 slots) use one
// chain with column 0 applied in pairs (walk_chunk_compact).  A block is 2^B
// steps, B = PERM_GENERIC_B.  Each generic_<arith>.cu file instantiates these
// templates for one arithmetic and every NMAX bucket; the build compiles the
// files in parallel.
#pragma once

// (The host emulation tests compile the walk part of this file as host C++;
// they leave out the CUDA runtime and the launchers.)
#ifndef PERM_HOST_EMULATION
#include <cuda_runtime.h>

#include "kernels.hpp"
#endif
#include "core.cuh"

#ifndef PERM_GENERIC_B
#define PERM_GENERIC_B 5
#endif

// Resident 256-thread blocks per SM the walk kernels are compiled for by
// default (their register budget): 2 -> 128 registers, 3 -> 80.  Narrow exact
// rings take three (WalkMinBlocks below).
#ifndef PERM_GENERIC_MIN_BLOCKS
#define PERM_GENERIC_MIN_BLOCKS 2
#endif

namespace pk {

// Register-slot access by a run-time index: a switch whose cases name x[k]
// with a compile-time k, so x stays in registers.  The switch argument is
// warp-uniform (a bit of a column mask, a group boundary), so it is a uniform
// jump, and only the slots a column really touches cost an arithmetic
// instruction.  The compiler cannot prove the arguments uniform; the walk's
// once-per-block warp vote (core.cuh) is the reconvergence point that keeps
// the lanes together.
// (A predicated loop over all NMAX slots would issue NMAX FP64 instructions
// per flip whatever the mask: on GB300 a predicated-off DFMA costs the FP64
// pipe as much as an executed one, and FP64 issues at 1/64 of FP32.)
//
// Contiguous slot ranges -- a row group, column 0's rows, the rows a column
// touches first -- take one jump into a descending ladder of cases that fall
// through to the end of the range, instead of one jump per slot.
#define PERM_SLOT_CASES(F)                                                                              \
    F(0) F(1) F(2) F(3) F(4) F(5) F(6) F(7) F(8) F(9) F(10) F(11) F(12) F(13) F(14) F(15) F(16) F(17)   \
    F(18) F(19) F(20) F(21) F(22) F(23) F(24) F(25) F(26) F(27) F(28) F(29) F(30) F(31) F(32) F(33)     \
    F(34) F(35) F(36) F(37) F(38) F(39) F(40) F(41) F(42) F(43) F(44) F(45) F(46) F(47)
#define PERM_SLOT_CASES_DOWN(F)                                                                         \
    F(47) F(46) F(45) F(44) F(43) F(42) F(41) F(40) F(39) F(38) F(37) F(36) F(35) F(34) F(33) F(32)     \
    F(31) F(30) F(29) F(28) F(27) F(26) F(25) F(24) F(23) F(22) F(21) F(20) F(19) F(18) F(17) F(16)    \
    F(15) F(14) F(13) F(12) F(11) F(10) F(9) F(8) F(7) F(6) F(5) F(4) F(3) F(2) F(1) F(0)

// Column masks: 32 bits are enough below 33 slots (one find-first-set per slot).
template <int NMAX> struct SlotMask { typedef u64 T; static __device__ __forceinline__ int low(T v) { return ctz64(v); } };
template <> struct SlotMask<16> { typedef u32 T; static __device__ __forceinline__ int low(T v) { return __ffs((int)v) - 1; } };
template <> struct SlotMask<32> { typedef u32 T; static __device__ __forceinline__ int low(T v) { return __ffs((int)v) - 1; } };

// Exact arithmetic with folded products: for matrices whose rows have
// absolute sums <= 127 every |x_i| is <= 127, so four consecutive factors
// multiply exactly in 32 bits (127^4 < 2^28) and one ring multiplication
// takes all four.  The fold blocks are fixed slot quadruples [4t, 4t+3].
template <int NL> struct ArithExactFold : ArithExact<NL> {};
template <class A> struct FoldOf { static constexpr bool v = false; };
template <int NL> struct FoldOf<ArithExactFold<NL>> { static constexpr bool v = true; };

template <int NMAX, class A>
struct GenericPol {
    static constexpr int NX = NMAX;
    static constexpr int Bv = PERM_GENERIC_B;
    // Two-state chains (core.cuh) where a group's product can be shared by
    // both chains (FP64); ring products cannot, so the exact walks keep one
    // chain and apply column 0 (walk_chunk_compact).  At 48 slots the second
    // chain's registers would spill x, so that bucket keeps one chain too.
    static constexpr bool kDual = A::kProdIsX && NMAX <= 32;
    static constexpr bool kUnrolledDual = false;   // the pairs of a block are a rolled loop
    static constexpr bool kAbs = true;             // sum|terms| is always kept
    static constexpr bool kZeroSpans = true;       // the two-state walk widens zero skips (core.cuh)
    typedef typename A::X X;
    typedef typename A::P P;
    typedef typename A::V V;
    typedef DevMat<NMAX, V, typename A::X0> M;
    typedef typename SlotMask<NMAX>::T Mask;

    const M *m;
    int abs_shift;      // sum|terms| is accumulated as sum|terms| 2^-abs_shift
    P Qh[NMAX + 1];     // chain levels >= B (dynamic index: local memory)
    P Bh[kDual ? NMAX + 1 : 1];   // the same levels of the column-0-on chain

    __device__ __forceinline__ GenericPol(const M *mat, int shift) : m(mat), abs_shift(shift) {}

    __device__ __forceinline__ int gbegin(int g) const { return ((const volatile unsigned char *)m->gbegin)[g]; }
    __device__ __forceinline__ int sbegin(int g) const { return ((const volatile unsigned char *)m->sbegin)[g]; }
    __device__ __forceinline__ Mask colmask(int j) const { return (Mask)((const volatile u64 *)m->colmask)[j]; }
    __device__ __forceinline__ const volatile V *colvals(int j) const {
        return m->val + ((const volatile unsigned short *)m->colptr)[j];
    }

    // x[i] = x[i] + s * v for a run-time slot i
    __device__ __forceinline__ static void add_slot(X (&x)[NX], int i, V v, int s) {
        switch (i) {
#define PERM_ADD_CASE(k)                                              \
    case k:                                                           \
        if constexpr (k < NMAX) x[k] = A::upd_rt(x[k], v, s);         \
        break;
            PERM_SLOT_CASES(PERM_ADD_CASE)
#undef PERM_ADD_CASE
        default: break;
        }
    }
    // q * x[b] * ... * x[e-1] (b < e), highest slot first
    __device__ __forceinline__ static P prod_range(const X (&x)[NX], int b, int e, P q) {
        if constexpr (FoldOf<A>::v) return prod_range_folded(x, b, e, q);
        switch (e) {
#define PERM_PROD_CASE(k)                                             \
    case k + 1:                                                       \
        if constexpr (k < NMAX) {                                     \
            q = A::mul(q, x[k]);                                      \
            if (k <= b) break;                                        \
        }                                                             \
        [[fallthrough]];
            PERM_SLOT_CASES_DOWN(PERM_PROD_CASE)
#undef PERM_PROD_CASE
        default: break;
        }
        return q;
    }
    // the same with the factors of each slot quadruple multiplied in 32 bits
    // first (FoldOf<A>): a quadruple starts at k = 4t+3 and folds at k = 4t
    // or where the range ends
    __device__ __forceinline__ static P prod_range_folded(const X (&x)[NX], int b, int e, P q) {
        int t = 1;
        switch (e) {
#define PERM_FPROD_CASE(k)                                            \
    case k + 1:                                                       \
        if constexpr (k < NMAX) {                                     \
            if constexpr (k % 4 == 3) t = x[k];                       \
            else t *= x[k];                                           \
            if constexpr (k % 4 == 0) {                               \
                q = A::mul(q, t);                                     \
                if (k <= b) break;                                    \
            } else if (k <= b) {                                      \
                q = A::mul(q, t);                                     \
                break;                                                \
            }                                                         \
        }                                                             \
        [[fallthrough]];
            PERM_SLOT_CASES_DOWN(PERM_FPROD_CASE)
#undef PERM_FPROD_CASE
        default: break;
        }
        return q;
    }
    // x[b] * ... * x[e-1] (b < e): one jump to the first factor, then the
    // ladder (no multiplication by 1)
    __device__ __forceinline__ static P prod_range1(const X (&x)[NX], int b, int e) {
        P t = A::one();
        switch (e) {
#define PERM_ENTRY_CASE(k)                                            \
    case k + 1:                                                       \
        if constexpr (k < NMAX) {                                     \
            t = x[k];                                                 \
            if (k <= b) return t;                                     \
        }                                                             \
        goto perm_step_##k;
            PERM_SLOT_CASES_DOWN(PERM_ENTRY_CASE)
#undef PERM_ENTRY_CASE
        default: return t;
        }
#define PERM_STEP_CASE(k)                                             \
    perm_step_##k:                                                    \
        if constexpr (k >= 1 && k <= NMAX) {                          \
            t = A::mul(t, x[k - 1]);                                  \
            if (k - 1 <= b) return t;                                 \
        }
        PERM_SLOT_CASES_DOWN(PERM_STEP_CASE)
#undef PERM_STEP_CASE
        return t;
    }
    // x[k] += s * w[k - b] for k in [b, e) (b < e), highest slot first
    __device__ __forceinline__ static void add_range(X (&x)[NX], int b, int e, const volatile V *w, int s) {
        switch (e) {
#define PERM_ADDR_CASE(k)                                             \
    case k + 1:                                                       \
        if constexpr (k < NMAX) {                                     \
            x[k] = A::upd_rt(x[k], w[k - b], s);                      \
            if (k <= b) break;                                        \
        }                                                             \
        [[fallthrough]];
            PERM_SLOT_CASES_DOWN(PERM_ADDR_CASE)
#undef PERM_ADDR_CASE
        default: break;
        }
    }

    // Column j: the rows it shares with earlier groups one slot at a time,
    // then its own group (the rows it touches first) as one range.
    __device__ __forceinline__ void flip_dyn(int j, X (&x)[NX], int s) {
        const int b = gbegin(j), e = gbegin(j + 1);
        Mask cm = colmask(j) & (Mask)((1ull << b) - 1);
        const volatile V *v = colvals(j);
        while (cm) {
            const int i = SlotMask<NMAX>::low(cm);
            cm &= cm - 1;
            add_slot(x, i, *v++, s);
        }
        if (b < e) add_range(x, b, e, v, s);
    }
    template <int J>
    __device__ __forceinline__ void flip_rt(X (&x)[NX], int s) { flip_dyn(J, x, s); }

    __device__ __forceinline__ P grp_dyn(int g, const X (&x)[NX], P q) const {
        const int b = gbegin(g), e = gbegin(g + 1);
        return b < e ? prod_range(x, b, e, q) : q;
    }

    // Steps l (even) and l+1 of a block, l+1 flipping column 0 with sign S
    // (+1 or -1, run time): both terms share Q_1 and differ only in column
    // 0's rows, the slots [0, |R_0|), whose values are the image's first
    // |R_0|.  One ladder multiplies the rows before the flip, applies it, and
    // multiplies after.
    __device__ __forceinline__ void pair_terms_rt(X (&x)[NX], P q1, typename A::Blk &blk, int S) {
        const volatile V *v = m->val;
        P p0 = q1, p1 = q1;
        if constexpr (FoldOf<A>::v) {
            int t0 = 1, t1 = 1;
            switch (gbegin(1)) {
#define PERM_RFPAIR_CASE(k)                                           \
    case k + 1:                                                       \
        if constexpr (k < NMAX) {                                     \
            const X xo = x[k];                                        \
            x[k] = A::upd_rt(xo, v[k], S);                            \
            if constexpr (k % 4 == 3) {                               \
                t0 = xo;                                              \
                t1 = x[k];                                            \
            } else {                                                  \
                t0 *= xo;                                             \
                t1 *= x[k];                                           \
            }                                                         \
            if constexpr (k % 4 == 0) {                               \
                p0 = A::mul(p0, t0);                                  \
                p1 = A::mul(p1, t1);                                  \
            }                                                         \
        }                                                             \
        [[fallthrough]];
                PERM_SLOT_CASES_DOWN(PERM_RFPAIR_CASE)
#undef PERM_RFPAIR_CASE
            default: break;
            }
        } else {
            switch (gbegin(1)) {
#define PERM_RPAIR_CASE(k)                                            \
    case k + 1:                                                       \
        if constexpr (k < NMAX) {                                     \
            p0 = A::mul(p0, x[k]);                                    \
            x[k] = A::upd_rt(x[k], v[k], S);                          \
            p1 = A::mul(p1, x[k]);                                    \
        }                                                             \
        [[fallthrough]];
                PERM_SLOT_CASES_DOWN(PERM_RPAIR_CASE)
#undef PERM_RPAIR_CASE
            default: break;
            }
        }
        A::template blk_add<1>(blk, p0);
        A::template blk_add<-1>(blk, p1);
        A::blk_abs(blk, p0, abs_shift);
        A::blk_abs(blk, p1, abs_shift);
    }
    // levels from..to of the single chain (Qh, local memory), from >= to,
    // each from the one above; returns level `to`
    __device__ __forceinline__ P rebuild(const X (&x)[NX], int from, int to) {
        P q = Qh[from + 1];
#pragma unroll 1
        for (int g = from; g >= to; --g) {
            q = grp_dyn(g, x, q);
            Qh[g] = q;
        }
        return q;
    }

    // qa *= x[k], qb *= x[k] + a_k0 for the rows k in [b, e) of column 0
    // (b < e), highest slot first; column 0's values are the image's first
    __device__ __forceinline__ void dual_range(const X (&x)[NX], int b, int e, P &qa, P &qb) const {
        const volatile V *v = m->val;
        switch (e) {
#define PERM_DUAL_CASE(k)                                             \
    case k + 1:                                                       \
        if constexpr (k < NMAX) {                                     \
            qa = A::mul(qa, x[k]);                                    \
            qb = A::mul(qb, A::template upd<1>(x[k], v[k]));          \
            if (k <= b) break;                                        \
        }                                                             \
        [[fallthrough]];
            PERM_SLOT_CASES_DOWN(PERM_DUAL_CASE)
#undef PERM_DUAL_CASE
        default: break;
        }
    }
    // level g of both chains from level g+1: group g, then S_g
    __device__ __forceinline__ void level2(int g, const X (&x)[NX], P qa_in, P qb_in, P &qa, P &qb) const {
        const int b = gbegin(g), e = gbegin(g + 1);
        if (b < e) {
            if constexpr (A::kProdIsX) {
                const P t = prod_range1(x, b, e);
                qa = A::mul(qa_in, t);
                qb = A::mul(qb_in, t);
            } else {
                qa = prod_range(x, b, e, qa_in);
                qb = prod_range(x, b, e, qb_in);
            }
        } else {
            qa = qa_in;
            qb = qb_in;
        }
        const int sb = sbegin(g), se = sbegin(g + 1);
        if (sb < se) dual_range(x, sb, se, qa, qb);
    }
    // both chains, all levels from the top down to B
    __device__ __forceinline__ void chain_init2(const X (&x)[NX], P &QA, P &QB) {
        const int top = m->top;
        P qa = A::one(), qb = A::one();
        for (int g = NMAX; g > top; --g) { Qh[g] = qa; Bh[g] = qb; }
        for (int g = top; g >= Bv; --g) {
            level2(g, x, qa, qb, qa, qb);
            Qh[g] = qa;
            Bh[g] = qb;
        }
        QA = qa;
        QB = qb;
    }
    // after a flip of column j >= B: levels j..B of both chains
    __device__ __forceinline__ void chain_hi2(int j, const X (&x)[NX], P &QA, P &QB) {
        P qa = Qh[j + 1], qb = Bh[j + 1];
        for (int g = j; g >= Bv; --g) {
            level2(g, x, qa, qb, qa, qb);
            Qh[g] = qa;
            Bh[g] = qb;
        }
        QA = qa;
        QB = qb;
    }

    // level L >= B of the chain(s) is zero (both chains for the two-state walk)
    __device__ __forceinline__ bool level_zero(int L) const {
        if constexpr (kDual) return A::is_zero(Qh[L]) && A::is_zero(Bh[L]);
        else return A::is_zero(Qh[L]);
    }

    // x = x0 + sum of the columns set in Gray code G (columns < n-1 only);
    // called by the whole warp, which visits the union of its lanes' columns
    __device__ __forceinline__ void init_x(X (&x)[NX], u64 G) {
#pragma unroll
        for (int i = 0; i < NMAX; ++i) x[i] = A::load_x0(m->x0, i);
        u64 U = warp_or64(G);
        while (U) {
            const int p = ctz64(U);
            U &= U - 1;
            flip_dyn(p, x, (int)((G >> p) & 1ull));
        }
    }
};

// The single-chain walk of the generic kernels (exact arithmetic, and FP64 at
// 48 slots), arranged so that each data-driven piece of code -- a column
// flip, a run of level rebuilds, the column-0 pair -- is inlined at one or two
// places only: every chain level lives in one local array, the 2^(B-1) pairs
// of a block are one rolled loop, and the column-0 sign is a run-time value.
// (Slot ladders inlined at a dozen call sites made the exact kernels wait on
// instruction fetch.)  Pair p of a block: the flip before it is column
// 1 + ctz(p) with sign bit 1 + ctz(p) of p (Theorem 1; bit B of the block
// start for column B-1), then steps 2p and 2p+1 differ by column 0 with sign
// + for even p.
template <int NMAX, class A>
__device__ __forceinline__ typename A::Acc walk_chunk_compact(GenericPol<NMAX, A> &pol, u64 q, int K, int zero_skip,
                                                              u64 &skipped) {
    constexpr int Bv = PERM_GENERIC_B;
    typedef typename A::X X;
    typedef typename A::P P;
    X x[NMAX];
    const u64 g0 = q << K;
    pol.init_x(x, g0 ^ (g0 >> 1));
    const int top = pol.m->top;
    for (int g = NMAX; g > top; --g) pol.Qh[g] = A::one();
    typename A::Acc acc = A::acc_zero();
    typename A::Blk mid = A::blk_zero();
    const u64 nblocks = 1ull << (K - Bv);
    for (u64 h = 0; h < nblocks; ++h) {
        if (h != 0 && (h & 7) == 0) {
            A::acc_merge(acc, mid);
            mid = A::blk_zero();
        }
        const u64 gb = g0 + (h << Bv);
        int from = top > Bv ? top : Bv;   // chunk start: every level down to B
        if (h != 0) {
            from = Bv + ctz64(h);
            pol.flip_dyn(from, x, ((gb >> (from + 1)) & 1ull) ? -1 : 1);
        }
        const P qB = pol.rebuild(x, from, Bv);
        const int s_mid = ((gb >> Bv) & 1ull) ? -1 : 1;
        // the vote is also the warp's reconvergence point after the
        // data-driven loops of the flips
        const bool all_zero = __all_sync(PERM_FULLMASK, A::is_zero(qB));
        if (zero_skip && all_zero) {
            // the block's net effect on x.  (This walk does not widen the skip
            // into zero spans: on the small exact matrices it serves, the
            // wider skip path cost more than the spans saved.)
            pol.flip_dyn(Bv - 1, x, s_mid);
            ++skipped;
            continue;
        }
        typename A::Blk blk = A::blk_zero();
#pragma unroll 1
        for (int p = 0; p < (1 << (Bv - 1)); ++p) {
            int lev = Bv - 1;
            if (p != 0) {
                lev = __ffs(p);   // 1 + ctz(p)
                const int s = (lev == Bv - 1) ? s_mid : (((p >> lev) & 1) ? -1 : 1);
                pol.flip_dyn(lev, x, s);
            }
            const P q1 = pol.rebuild(x, lev, 1);
            pol.pair_terms_rt(x, q1, blk, (p & 1) ? -1 : 1);
        }
        A::blk_accumulate(mid, blk);
    }
    A::acc_merge(acc, mid);
    return acc;
}

// The generic walk over any number of matrices (a single matrix is a batch
// of one).  Warps of a persistent grid take 32-chunk tasks from one counter;
// a task's matrix is found by binary search over the task ranges, and the
// warp stages that matrix's image in its own shared-memory slot (restaged
// only when the matrix changes).
template <int NMAX, class A>
__device__ __forceinline__ void generic_task_loop(const BatchArgs &ba, unsigned char *slot_raw) {
    typedef DevMat<NMAX, typename A::V, typename A::X0> M;
    const int lane = threadIdx.x & 31;
    M *slot = reinterpret_cast<M *>(slot_raw);
    int cached = -1;
    u64 skipped = 0;
    for (;;) {
        u64 task = 0;
        if (lane == 0) task = past_deadline(ba.timeout_ns, ba.deadline_word, ba.abort_flag) ? ~0ull : atomicAdd(ba.task_counter, 1ull);
        task = __shfl_sync(PERM_FULLMASK, task, 0);
        if (task >= ba.ntasks) break;
        int m = 0;
        if (lane == 0) {
            int lo = 0, hi = ba.nmat - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (ba.mats[mid].task_begin <= task) lo = mid; else hi = mid - 1;
            }
            m = lo;
        }
        m = __shfl_sync(PERM_FULLMASK, m, 0);
        const BatchMat bm = ba.mats[m];
        if (bm.image != cached) {
            __syncwarp();
            const uint4 *src = reinterpret_cast<const uint4 *>(
                reinterpret_cast<const unsigned char *>(ba.devmats) + (size_t)bm.image * 16);
            const int words = reinterpret_cast<const int *>(src)[3] / 16;   // the image's own size
            uint4 *dst = reinterpret_cast<uint4 *>(slot);
            for (int i = lane; i < words; i += 32) dst[i] = src[i];
            __syncwarp();
            cached = bm.image;
        }
        u64 q = bm.chunk_lo + (task - bm.task_begin) * 32ull + (u64)lane;
        const bool live = q < bm.chunk_hi;
        if (!live) q = bm.chunk_hi - 1;     // idle lanes shadow a real chunk to stay in step
        GenericPol<NMAX, A> pol(slot, bm.abs_shift);
        typename A::Acc acc;
        if constexpr (GenericPol<NMAX, A>::kDual)
            acc = walk_chunk_dual<GenericPol<NMAX, A>, A, PERM_GENERIC_B>(pol, q, bm.K, ba.zero_skip, skipped);
        else
            acc = walk_chunk_compact<NMAX, A>(pol, q, bm.K, ba.zero_skip, skipped);
        if (!live) acc = A::acc_zero();
#pragma unroll
        for (int d = 16; d >= 1; d >>= 1) acc = A::acc_add(acc, A::shfl_down(acc, d));
        if (lane == 0) A::acc_store(ba.task_out + (bm.out_offset + (task - bm.task_begin)) * (u64)A::ACC_WORDS, acc);
    }
    // the warp's skipped blocks (a skip is warp-wide: one count per warp block)
    if (ba.skip_counter && lane == 0 && skipped) atomicAdd(ba.skip_counter, skipped);
}

// Resident blocks the walk kernel is compiled for: exact rings of up to 96
// bits at 32 slots, and up to 160 bits at 16, fit 80 registers without
// spilling, so they run three blocks (24 warps) per SM; the rest two.
template <class A> struct LimbsOf { static constexpr int v = 0; };
template <int NL> struct LimbsOf<ArithExact<NL>> { static constexpr int v = NL; };
template <int NL> struct LimbsOf<ArithExactFold<NL>> { static constexpr int v = NL; };
// Double-double walks hold two doubles per slot and get the whole register
// file of one block.
template <class A> struct IsDD { static constexpr bool v = false; };
template <> struct IsDD<ArithDD> { static constexpr bool v = true; };
template <int NMAX, class A> struct WalkMinBlocks {
    static constexpr int L = LimbsOf<A>::v;
    static constexpr int v = IsDD<A>::v ? 1
                             : (L > 0 && ((NMAX == 16 && L <= 5) || (NMAX == 32 && L <= 3))) ? 3
                                                                                             : PERM_GENERIC_MIN_BLOCKS;
};

template <int NMAX, class A>
__global__ void __launch_bounds__(256, WalkMinBlocks<NMAX, A>::v) k_walk_generic(BatchArgs ba) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5;
    generic_task_loop<NMAX, A>(ba, smem_raw + (size_t)warp * ba.slot_bytes);
}

// Tiny matrices: one thread per Gray index, x built from scratch.
template <int NMAX, class A>
__global__ void __launch_bounds__(256) k_direct_generic(const DevMat<NMAX, typename A::V, typename A::X0> *m, u64 g_lo,
                                                        u64 g_hi, u64 *block_out, int abs_shift) {
    typedef typename A::X X;
    const u64 g = g_lo + (u64)blockIdx.x * blockDim.x + threadIdx.x;
    typename A::Acc acc = A::acc_zero();
    if (g < g_hi) {
        X x[NMAX];
#pragma unroll
        for (int i = 0; i < NMAX; ++i) x[i] = A::load_x0(m->x0, i);
        u64 G = g ^ (g >> 1);
        while (G) {
            const int p = ctz64(G);
            G &= G - 1;
            const u64 cm = m->colmask[p];
            int k = m->colptr[p];
#pragma unroll
            for (int i = 0; i < NMAX; ++i)
                if ((cm >> i) & 1ull) x[i] = A::upd_rt(x[i], m->val[k++], 1);
        }
        typename A::P q = A::one();
#pragma unroll
        for (int i = 0; i < NMAX; ++i)
            if (i < m->n) q = A::mul(q, x[i]);
        typename A::Blk b = A::blk_zero();
        if (g & 1ull) A::template blk_add<-1>(b, q); else A::template blk_add<1>(b, q);
        A::blk_abs(b, q, abs_shift);
        A::acc_merge(acc, b);
    }
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) acc = A::acc_add(acc, A::shfl_down(acc, d));
    __shared__ u64 sh[8 * 6];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) A::acc_store(sh + warp * A::ACC_WORDS, acc);
    __syncthreads();
    if (warp == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        acc = lane < nw ? A::acc_load(sh + lane * A::ACC_WORDS) : A::acc_zero();
#pragma unroll
        for (int d = 16; d >= 1; d >>= 1) acc = A::acc_add(acc, A::shfl_down(acc, d));
        if (lane == 0) A::acc_store(block_out + (u64)blockIdx.x * A::ACC_WORDS, acc);
    }
}

}  // namespace pk

#ifndef PERM_HOST_EMULATION
namespace perm {

template <int NMAX, class A>
static cudaError_t launch_walk_t(const pk::BatchArgs &ba, int grid, int block, cudaStream_t st) {
    const size_t smem = (size_t)(block / 32) * ba.slot_bytes;
    cudaError_t e = cudaFuncSetAttribute(pk::k_walk_generic<NMAX, A>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    pk::k_walk_generic<NMAX, A><<<grid, block, smem, st>>>(ba);
    return cudaGetLastError();
}

template <int NMAX, class A>
static cudaError_t launch_direct_t(const void *devmat, uint64_t g_lo, uint64_t g_hi, uint64_t *out, int grid,
                                   int block, cudaStream_t st, int abs_shift) {
    pk::k_direct_generic<NMAX, A><<<grid, block, 0, st>>>(
        reinterpret_cast<const pk::DevMat<NMAX, typename A::V, typename A::X0> *>(devmat), g_lo, g_hi,
        reinterpret_cast<unsigned long long *>(out), abs_shift);
    return cudaGetLastError();
}

template <int NMAX, class A>
static cudaError_t attr_walk_t(cudaFuncAttributes *attr) {
    return cudaFuncGetAttributes(attr, pk::k_walk_generic<NMAX, A>);
}

template <int NMAX, class A>
static cudaError_t occ_walk_t(int block, size_t slot_bytes, int *blocks_per_sm) {
    const size_t smem = (size_t)(block / 32) * slot_bytes;
    cudaError_t e = cudaFuncSetAttribute(pk::k_walk_generic<NMAX, A>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, pk::k_walk_generic<NMAX, A>, block, smem);
}

template <int NMAX, class A>
static GenericFns make_fns() {
    GenericFns f;
    f.walk = launch_walk_t<NMAX, A>;
    f.direct = launch_direct_t<NMAX, A>;
    f.attr = attr_walk_t<NMAX, A>;
    f.occ = occ_walk_t<NMAX, A>;
    f.block_log2 = PERM_GENERIC_B;
    f.devmat_bytes = sizeof(pk::DevMat<NMAX, typename A::V, typename A::X0>);   // capacity of a dense image
    return f;
}

}  // namespace perm
#endif  // PERM_HOST_EMULATION

// Defines perm::generic_fns_<NAME>(nmax) for one arithmetic.
#define PERM_GENERIC_UNIT(NAME, ARITH)                                   \
    namespace perm {                                                     \
    GenericFns generic_fns_##NAME(int nmax) {                            \
        switch (nmax) {                                                  \
        case 16: return make_fns<16, ARITH>();                           \
        case 32: return make_fns<32, ARITH>();                           \
        case 48: return make_fns<48, ARITH>();                           \
        default: return GenericFns();                                    \
        }                                                                \
    }                                                                    \
    }

// Defines perm::generic_fns_<NAME>(nmax, fold) for one exact ring width,
// with (fold = 1) and without folded products.
#define PERM_GENERIC_EXACT_UNIT(NAME, NL)                                \
    namespace perm {                                                     \
    GenericFns generic_fns_##NAME(int nmax, int fold) {                  \
        if (fold) {                                                      \
            switch (nmax) {                                              \
            case 16: return make_fns<16, pk::ArithExactFold<NL>>();      \
            case 32: return make_fns<32, pk::ArithExactFold<NL>>();      \
            case 48: return make_fns<48, pk::ArithExactFold<NL>>();      \
            default: return GenericFns();                                \
            }                                                            \
        }                                                                \
        switch (nmax) {                                                  \
        case 16: return make_fns<16, pk::ArithExact<NL>>();              \
        case 32: return make_fns<32, pk::ArithExact<NL>>();              \
        case 48: return make_fns<48, pk::ArithExact<NL>>();              \
        default: return GenericFns();                                    \
        }                                                                \
    }                                                                    \
    }
