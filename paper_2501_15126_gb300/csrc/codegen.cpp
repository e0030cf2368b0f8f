// codegen.cpp -- matrix-specific kernel generation and runtime compilation.
//
// For one ordered matrix the generator writes CUDA C++ in which (Sec. III-B):
//   * every row of x in registers is a named slot x[s] with a compile-time
//     index, so the register-allocation condition of Sec. III-A holds;
//   * the inclusion/exclusion of column j (Listing 2) is a list of updates of
//     those slots by literal values (hex-float literals: exact), with the
//     sign either a compile-time constant (inside the unrolled block) or a
//     per-lane +-1 (the one divergent case of Lemma 1);
//   * the product is rebuilt through the chain of group products (core.cuh),
//     the generalisation of Listings 3-5;
//   * rows beyond the first k slots live in global memory at
//     x[(slot - k) * nthreads + tid] (Listing 4's coalesced layout), touched
//     only by columns >= c (Algorithm 4).
// The text is compiled by NVRTC for sm_103a and loaded through the CUDA
// driver API; kernels are cached by their source text for the life of the
// process.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <sstream>
#include <string>
#include <unordered_map>
#include <vector>

#include <cuda.h>
#include <cuda_runtime.h>
#include <nvrtc.h>

#include "codegen.hpp"
#include "plan.hpp"

// Embedded copies of core.cuh and devmat.h (generated at build time).
extern const char *perm_embedded_core_cuh;
extern const char *perm_embedded_devmat_h;

namespace perm {

namespace {

// Steps per unrolled block, log2.  FP64 walks take longer blocks: the block
// start (run-time flip, chain rebuild, vote) is then spread over more steps
// (the n=36 FP64 walk: 370.9 ms at 2^5, 365.5 at 2^6, 361.5 at 2^7), and
// their compile time grows little (0.64 -> 0.76 s).  Exact walks keep 2^5: at
// 2^6 their NVRTC time grows by half and some need all 255 registers, and at
// 2^4 the n=48 band walk is 19 % slower (5.95 against 5.00 ms per 2^30
// steps).  FP64 walks where most terms are zero keep 2^5 too: their zero skip
// starts at a block (the d_ss shape: 1.66e12 Gray steps/s at 2^5, 0.98e12 at
// 2^7).  Exact walks where nearly every term is zero (over 95 % of the
// sampled ones) but without zero spans (a warp's lanes rarely share a zero
// row, so only single blocks are skipped, where every lane's products are
// zero at once) take 2^4: a finer skip and half the unrolled body (the
// mycielskian6 shape, 99.6 % zero terms: 235 against 306 ms per 2^36 steps,
// 43 % of the blocks skipped against 38 %).  The n=48 band, 74 % zero terms,
// skips no block and keeps 2^5.
constexpr int kCodegenBlockLog2F64 = 7;
constexpr int kCodegenBlockLog2ZeroHeavy = 5;
constexpr int kCodegenBlockLog2Exact = 5;
constexpr int kCodegenBlockLog2ZeroBlocks = 4;
constexpr int kCodegenBlock = 256;

// ------------------------------------------------------------------ driver API via the runtime
struct Driver {
    CUresult (*moduleLoadData)(CUmodule *, const void *) = nullptr;
    CUresult (*moduleGetFunction)(CUfunction *, CUmodule, const char *) = nullptr;
    CUresult (*launchKernel)(CUfunction, unsigned, unsigned, unsigned, unsigned, unsigned, unsigned, unsigned,
                             CUstream, void **, void **) = nullptr;
    CUresult (*funcGetAttribute)(int *, CUfunction_attribute, CUfunction) = nullptr;
    CUresult (*occupancy)(int *, CUfunction, int, size_t) = nullptr;
    CUresult (*getErrorString)(CUresult, const char **) = nullptr;
    CUresult (*moduleUnload)(CUmodule) = nullptr;
    CUresult (*funcSetAttribute)(CUfunction, CUfunction_attribute, int) = nullptr;
    bool ok = false;
};

template <class F>
static bool entry(const char *name, F &fp) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion(name, &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !p)
        return false;
    fp = reinterpret_cast<F>(p);
    return true;
}

Driver &driver() {
    static Driver d;
    static std::once_flag once;
    std::call_once(once, [] {
        d.ok = entry("cuModuleLoadData", d.moduleLoadData) && entry("cuModuleGetFunction", d.moduleGetFunction) &&
               entry("cuLaunchKernel", d.launchKernel) && entry("cuFuncGetAttribute", d.funcGetAttribute) &&
               entry("cuOccupancyMaxActiveBlocksPerMultiprocessor", d.occupancy) &&
               entry("cuGetErrorString", d.getErrorString) && entry("cuModuleUnload", d.moduleUnload) &&
               entry("cuFuncSetAttribute", d.funcSetAttribute);
    });
    return d;
}

std::string cu_err(CUresult r) {
    const char *s = nullptr;
    if (driver().getErrorString) driver().getErrorString(r, &s);
    return s ? s : "unknown driver error";
}

// ------------------------------------------------------------------ source emission
// Resident 256-thread blocks per SM that the generated kernel is compiled for
// (its register budget: 1 -> 255 registers, 2 -> 128, 3 -> 85).  FP64 walks
// of 2^30 steps and more (those the automatic engine generates kernels for)
// take one block: eight warps per SM keep the FP64 pipe as busy as sixteen,
// and 255 registers hold x and both chains without spilling (the n=36
// workload: 224 registers, no spills, 359.9 ms per permanent against 361.8 ms
// at 128 registers with 152 bytes of spills; the bcsstk01 and mesh1e1
// shapes 1.1 and 1.4 % faster, kernels that fit 128 registers unchanged).
// Shorter FP64 walks keep two blocks (an n=28 walk, 2^27 steps: 2.6 %
// slower with half the warps to share its tasks), and so do exact walks,
// which are bound by instruction issue and need the warps (the n=48 band:
// 5.86 ms at one block against 5.00 at two).  CodeGen-PureReg keeps two
// blocks, as measured in the ablation.  PERM_CODEGEN_MIN_BLOCKS overrides.
int codegen_min_blocks(const perm_plan_s &P) {
    const char *e = std::getenv("PERM_CODEGEN_MIN_BLOCKS");
    if (e) {
        const int v = std::atoi(e);
        if (v >= 1 && v <= 8) return v;
    }
    return P.arith == 0 && !P.pure_reg && P.len() >= (1ull << 30) ? 1 : 2;
}
// PERM_CODEGEN_NO_FOLD=1: exact kernels multiply every row into the ring on
// its own (no 32-bit folding), as they did before folding was introduced.
bool no_fold_env() {
    const char *e = std::getenv("PERM_CODEGEN_NO_FOLD");
    return e && std::atoi(e) == 1;
}
std::string lit(const perm_plan_s &P, double v) {
    char buf[64];
    if (P.arith == 0) {
        std::snprintf(buf, sizeof buf, "%a", v);
        std::string s(buf);
        return v < 0 ? "(" + s + ")" : s;
    }
    std::snprintf(buf, sizeof buf, "%lld", (long long)v);
    std::string s(buf);
    return v < 0 ? "(" + s + ")" : s;
}

struct Emitter {
    const perm_plan_s &P;
    int n, k, c, k2;
    int min_blocks;   // __launch_bounds__ minimum resident blocks per SM (register budget)
    std::ostringstream o;
    Emitter(const perm_plan_s &p, int mb) : P(p), n(p.m.n), k(p.k), c(p.c), k2(p.k2), min_blocks(mb) {}

    // value of ordered column p at slot s (doubled on the exact path)
    bool has(int p, int s) const { return (P.L.colmask[p] >> s) & 1ull; }
    double value(int p, int s) const {
        const int r = P.L.row_order[s], col = P.L.col_order[p];
        return P.arith == 0 ? P.m.fval(r, col) : 2.0 * (double)P.m.ival(r, col);
    }
    std::string slot(int s) const {
        if (s < k) return "x[" + std::to_string(s) + "]";
        if (s < k + k2) return "xs[" + std::to_string(s - k) + "u * 256u]";   // the block's shared tier
        return "xg[" + std::to_string(s - k - k2) + "ull * stride]";
    }
    // one update of slot s by column p; mode 1/-1 = static sign, 0 = runtime s
    void update(int p, int s, int mode, const char *ind) {
        const std::string v = lit(P, value(p, s));
        const std::string x = slot(s);
        if (s < k) {
            if (mode > 0) o << ind << x << " += " << v << ";\n";
            else if (mode < 0) o << ind << x << " -= " << v << ";\n";
            else o << ind << x << " = A::upd_rt(" << x << ", " << v << ", s);\n";
        } else {
            o << ind << "{ X t = " << x << "; ";
            if (mode > 0) o << "t += " << v << "; ";
            else if (mode < 0) o << "t -= " << v << "; ";
            else o << "t = A::upd_rt(t, " << v << ", s); ";
            o << x << " = t; }\n";
        }
    }
    void column(int p, int mode, const char *ind) {
        for (int s = 0; s < n; ++s)
            if (has(p, s)) update(p, s, mode, ind);
    }
    // q *= the rows of group g.  Exact walks multiply runs of rows in 32 bits
    // first while the product of the rows' absolute sums (which bound |x_i|
    // at every Gray index) stays below 2^31, then fold each run into the ring
    // with one multiplication.
    void group_product(int g, const char *ind) { product_range(P.L.group_begin[g], P.L.group_begin[g + 1], ind); }
    // q *= the slots [b, e), folded in 32 bits on the exact path
    void product_range(int b, int e, const char *ind) {
        if (P.arith == 0 || no_fold_env()) {
            for (int s = b; s < e; ++s) o << ind << "q = A::mul(q, " << slot(s) << ");\n";
            return;
        }
        int s = b;
        while (s < e) {
            double bound = row_abs_sum(s);
            int t = s + 1;
            while (t < e && bound * row_abs_sum(t) < 2147483647.0) bound *= row_abs_sum(t++);
            if (t == s + 1) {
                o << ind << "q = A::mul(q, " << slot(s) << ");\n";
            } else {
                o << ind << "q = A::mul(q, " << slot(s);
                for (int u = s + 1; u < t; ++u) o << " * " << slot(u);
                o << ");\n";
            }
            s = t;
        }
    }
    double row_abs_sum(int s) const {
        const int r = P.L.row_order[s];
        double a = 0.0;
        for (int j = 0; j < n; ++j) a += std::fabs(P.m.fval(r, j));
        return std::max(a, 1.0);
    }
    // two-state chains: level g holds group g and S_g (column 0's rows next
    // touched by column g)
    bool level_nonempty(int g) const {
        return P.L.group_begin[g + 1] > P.L.group_begin[g] || P.L.s_begin[g + 1] > P.L.s_begin[g];
    }
    std::vector<int> high_levels2(int B) const {
        std::vector<int> v;
        for (int g = n - 1; g >= B; --g)
            if (level_nonempty(g)) v.push_back(g);
        return v;
    }
    // qa = ain * prod_{group g} x * prod_{S_g} x, qb = bin * prod_{group g} x * prod_{S_g} (x + a_0)
    void level2_code(int g, const std::string &ain, const std::string &bin, const char *ind) {
        const int b = P.L.group_begin[g], e = P.L.group_begin[g + 1];
        if (b < e) {
            o << ind << "{\n" << ind << "    P t = " << slot(b) << ";\n";
            for (int s = b + 1; s < e; ++s) o << ind << "    t = t * " << slot(s) << ";\n";
            o << ind << "    qa = " << ain << " * t;\n" << ind << "    qb = " << bin << " * t;\n" << ind << "}\n";
        } else if (ain != "qa") {
            o << ind << "qa = " << ain << ";\n" << ind << "qb = " << bin << ";\n";
        }
        for (int s = P.L.s_begin[g]; s < P.L.s_begin[g + 1]; ++s) {
            o << ind << "qa = qa * " << slot(s) << ";\n";
            o << ind << "qb = qb * (" << slot(s) << " + " << lit(P, value(0, s)) << ");\n";
        }
    }
    // the level functions, start and rebuild of the two-state chains
    void emit_dual(int B) {
        const std::vector<int> hi2 = high_levels2(B);
        o << "    template <int M> __device__ __forceinline__ void level2c(const X (&x)[NX], P qa_in, P qb_in, P &qa, P &qb) const {\n";
        for (int g = 1; g < B; ++g) {
            o << "        " << (g > 1 ? "else " : "") << "if constexpr (M == " << g << ") {\n";
            if (g < n) level2_code(g, "qa_in", "qb_in", "            ");
            else o << "            qa = qa_in;\n            qb = qb_in;\n";
            o << "        }\n";
        }
        o << "    }\n";
        o << "    __device__ __forceinline__ void level2(int M, const X (&x)[NX], P qa_in, P qb_in, P &qa, P &qb) const {\n";
        o << "        switch (M) {\n";
        for (int g = 1; g < B; ++g) o << "        case " << g << ": level2c<" << g << ">(x, qa_in, qb_in, qa, qb); break;\n";
        o << "        default: qa = qa_in; qb = qb_in; break;\n        }\n    }\n";
        o << "    __device__ __forceinline__ void chain_init2(const X (&x)[NX], P &QA, P &QB) {\n";
        o << "        P qa = A::one(), qb = A::one();\n";
        for (int g : hi2) {
            level2_code(g, "qa", "qb", "        ");
            o << "        QA" << g << " = qa;\n        QB" << g << " = qb;\n";
        }
        o << "        QA = qa;\n        QB = qb;\n    }\n";
        auto above2 = [&](int g) -> int {
            for (int h = g + 1; h < n; ++h)
                if (h >= B && level_nonempty(h)) return h;
            return -1;
        };
        o << "    __device__ __forceinline__ void chain_hi2(int j, const X (&x)[NX], P &QA, P &QB) {\n";
        o << "        P qa, qb;\n        switch (j) {\n";
        for (int j = B; j < n - 1; ++j) {
            const int a = above2(j);
            if (a >= 0) o << "        case " << j << ": qa = QA" << a << "; qb = QB" << a << "; break;\n";
            else o << "        case " << j << ": qa = A::one(); qb = A::one(); break;\n";
        }
        o << "        default: qa = A::one(); qb = A::one(); break;\n        }\n";
        o << "        switch (j) {\n";
        for (int j = n - 2; j >= B; --j) {
            o << "        case " << j << ":\n";
            if (level_nonempty(j)) {
                level2_code(j, "qa", "qb", "            ");
                o << "            QA" << j << " = qa;\n            QB" << j << " = qb;\n";
            }
            o << "            [[fallthrough]];\n";
        }
        o << "        default: break;\n        }\n";
        o << "        QA = qa;\n        QB = qb;\n    }\n";
    }

    // nonempty chain levels >= B, descending
    std::vector<int> high_levels(int B) const {
        std::vector<int> v;
        for (int g = n - 1; g >= B; --g)
            if (P.L.group_begin[g + 1] > P.L.group_begin[g]) v.push_back(g);
        return v;
    }

    std::string emit() {
        const int B = codegen_block_log2(P);
        const std::vector<int> hi = high_levels(B);
        o << "// generated: permanent walk for one " << n << "x" << n << " matrix\n";
        o << "// order=" << P.L.ordering << " reg_rows(k)=" << k << " reg_cols(c)=" << c << " B=" << B << "\n";
        o << "#include \"core.cuh\"\n\nnamespace pk {\n";
        if (P.arith == 0) o << "typedef ArithF64 A;\n";
        else o << "typedef ArithExact<" << P.limbs << "> A;\n";
        o << "struct GenPol {\n";
        o << "    static constexpr int NX = " << std::max(k, 1) << ";\n";
        o << "    static constexpr bool kPaired = " << (P.arith == 0 && !P.pure_reg ? "true" : "false") << ";\n";
        o << "    static constexpr bool kDual = " << (P.dual ? "true" : "false") << ";\n";
        o << "    static constexpr bool kUnrolledDual = true;\n";
        o << "    typedef A::X X;\n    typedef A::P P;\n";
        o << "    X *xg;\n    unsigned long long stride;\n    X *xs;\n";
        // sum|terms| is accumulated as sum|terms| 2^-abs_shift (core.cuh); the
        // paired step scales its column-0 products by 2^-SH0 and Q_1 by the rest
        o << "    static constexpr int abs_shift = " << (P.arith == 0 ? P.abs_shift : 0) << ";\n";
        o << "    static constexpr bool kAbs = " << (P.want_abs ? "true" : "false") << ";\n";
        o << "    static constexpr bool kZeroSpans = " << (P.zero_spans ? "true" : "false") << ";\n";
        if (P.dual) {
            for (int g : high_levels2(B)) o << "    P QA" << g << ", QB" << g << ";\n";
        } else if (!P.pure_reg) {
            for (int g : hi) o << "    P Q" << g << ";\n";
        }
        // level L >= B of the chain(s) is zero: the stored level at the first
        // nonempty group >= L (the zero spans of core.cuh)
        o << "    __device__ __forceinline__ bool level_zero(int L) const {\n";
        if (!P.pure_reg && P.zero_spans) {
            o << "        switch (L) {\n";
            for (int L = B; L < n; ++L) {
                int g = -1;
                for (int h = L; h < n && g < 0; ++h)
                    if (P.dual ? level_nonempty(h) : P.L.group_begin[h + 1] > P.L.group_begin[h]) g = h;
                if (g < 0) continue;
                if (P.dual)
                    o << "        case " << L << ": return A::is_zero(QA" << g << ") && A::is_zero(QB" << g << ");\n";
                else
                    o << "        case " << L << ": return A::is_zero(Q" << g << ");\n";
            }
            o << "        default: break;\n        }\n";
        }
        o << "        return false;\n    }\n";
        // flips inside the unrolled block (static column, static or runtime sign)
        o << "    template <int J, int S> __device__ __forceinline__ void flip(X (&x)[NX]) {\n";
        for (int p = 0; p < B && p < n - 1; ++p) {
            o << "        " << (p ? "else " : "") << "if constexpr (J == " << p << ") {\n";
            o << "            if constexpr (S > 0) {\n";
            column(p, 1, "                ");
            o << "            } else {\n";
            column(p, -1, "                ");
            o << "            }\n        }\n";
        }
        o << "    }\n";
        o << "    template <int J> __device__ __forceinline__ void flip_rt(X (&x)[NX], int s) {\n";
        for (int p = 0; p < B && p < n - 1; ++p) {
            o << "        " << (p ? "else " : "") << "if constexpr (J == " << p << ") {\n";
            column(p, 0, "            ");
            o << "        }\n";
        }
        o << "    }\n";
        // a flip chosen at run time (block boundaries, start vectors)
        o << "    __device__ __forceinline__ void flip_dyn(int j, X (&x)[NX], int s) {\n";
        o << "        switch (j) {\n";
        for (int p = 0; p < n - 1; ++p) {
            o << "        case " << p << ":\n";
            column(p, 0, "            ");
            o << "            break;\n";
        }
        o << "        default: break;\n        }\n    }\n";
        // paired steps (FP64): D = prod_{R_0} x - prod_{R_0} (x + S a_0), the
        // column-0 flip applied, Q_1 * D returned.  R_0 = column 0's rows = the
        // first slots.
        // The two terms' magnitudes |Q_1| (|prod_{R_0} x| + |prod_{R_0} (x + S a_0)|)
        // come back in FP32 through fa: integer and FP32 instructions only.
        if (P.arith == 0 && P.want_abs) {
            const int r0 = P.L.group_begin[1] - P.L.group_begin[0];
            double l0 = 0.0;   // log2 bound of a product over R_0
            for (int s2 = 0; s2 < r0; ++s2) l0 += std::log2(std::max(row_abs_sum(s2) / 2.0, 1e-300));
            const int sh0 = (int)std::ceil(l0) - 60;
            const std::string f1 = "abs_scaled_f32(q1, abs_shift - (" + std::to_string(sh0) + "))";
            const std::string sh = std::to_string(sh0);
            o << "    template <int S> __device__ __forceinline__ P pair(X (&x)[NX], P q1, float &fa) {\n";
            if (r0 == 1) {
                const std::string v = lit(P, value(0, 0));
                o << "        const X xo = x[0];\n";
                o << "        if constexpr (S > 0) x[0] += " << v << "; else x[0] -= " << v << ";\n";
                o << "        fa = " << f1 << " * (abs_scaled_f32(xo, " << sh << ") + abs_scaled_f32(x[0], " << sh
                  << "));\n";
                o << "        if constexpr (S > 0) return q1 * -" << v << "; else return q1 * " << v << ";\n";
            } else {
                o << "        P px = x[0];\n";
                for (int s2 = 1; s2 < r0 - 1; ++s2) o << "        px = px * x[" << s2 << "];\n";
                o << "        const X xl = x[" << r0 - 1 << "];\n";
                o << "        if constexpr (S > 0) {\n";
                for (int s2 = 0; s2 < r0; ++s2) o << "            x[" << s2 << "] += " << lit(P, value(0, s2)) << ";\n";
                o << "        } else {\n";
                for (int s2 = 0; s2 < r0; ++s2) o << "            x[" << s2 << "] -= " << lit(P, value(0, s2)) << ";\n";
                o << "        }\n";
                o << "        P py = x[0];\n";
                for (int s2 = 1; s2 < r0; ++s2) o << "        py = py * x[" << s2 << "];\n";
                o << "        fa = " << f1 << " * (abs_scaled_f32(px, " << sh << ") * abs_scaled_f32(xl, 0) + "
                  << "abs_scaled_f32(py, " << sh << "));\n";
                o << "        return q1 * fma(px, xl, -py);\n";
            }
            o << "    }\n";
        } else if (P.arith == 0) {   // the same without the magnitudes
            const int r0 = P.L.group_begin[1] - P.L.group_begin[0];
            o << "    template <int S> __device__ __forceinline__ P pair(X (&x)[NX], P q1, float &fa) {\n";
            o << "        fa = 0.f;\n";
            if (r0 == 1) {
                const std::string v = lit(P, value(0, 0));
                o << "        if constexpr (S > 0) { x[0] += " << v << "; return q1 * -" << v << "; }\n";
                o << "        else { x[0] -= " << v << "; return q1 * " << v << "; }\n";
            } else {
                o << "        P px = x[0];\n";
                for (int s2 = 1; s2 < r0 - 1; ++s2) o << "        px = px * x[" << s2 << "];\n";
                o << "        const X xl = x[" << r0 - 1 << "];\n";
                o << "        if constexpr (S > 0) {\n";
                for (int s2 = 0; s2 < r0; ++s2) o << "            x[" << s2 << "] += " << lit(P, value(0, s2)) << ";\n";
                o << "        } else {\n";
                for (int s2 = 0; s2 < r0; ++s2) o << "            x[" << s2 << "] -= " << lit(P, value(0, s2)) << ";\n";
                o << "        }\n";
                o << "        P py = x[0];\n";
                for (int s2 = 1; s2 < r0; ++s2) o << "        py = py * x[" << s2 << "];\n";
                o << "        return q1 * fma(px, xl, -py);\n";
            }
            o << "    }\n";
        } else {
            o << "    template <int S> __device__ __forceinline__ P pair(X (&x)[NX], P q1, float &fa) { fa = 0.f; return q1; }\n";
        }
        // group products of the low levels
        o << "    template <int M> __device__ __forceinline__ P grp(const X (&x)[NX], P q) const {\n";
        if (P.pure_reg) {
            // the paper's CodeGen-PureReg scheme: the product of all n rows at every step
            o << "        if constexpr (M == 0) {\n            q = A::one();\n";
            product_range(0, n, "            ");
            o << "        }\n        return q;\n    }\n";
        }
        for (int g = 0; g < B && !P.pure_reg; ++g) {
            o << "        " << (g ? "else " : "") << "if constexpr (M == " << g << ") {\n";
            if (g < n) group_product(g, "            ");
            o << "        }\n";
        }
        if (!P.pure_reg) o << "        return q;\n    }\n";
        // start vector
        o << "    __device__ __forceinline__ void init_x(X (&x)[NX], unsigned long long G) {\n";
        const int last = P.L.col_order[n - 1];
        for (int s = 0; s < n; ++s) {
            const int r = P.L.row_order[s];
            double x0;
            if (P.arith == 0) {
                double rowsum = 0.0;
                for (int j = 0; j < n; ++j) rowsum += P.m.fval(r, j);
                x0 = P.m.fval(r, last) - rowsum / 2.0;
            } else {
                int64_t rowsum = 0;
                for (int j = 0; j < n; ++j) rowsum += P.m.ival(r, j);
                x0 = (double)(2 * P.m.ival(r, last) - rowsum);
            }
            o << "        " << slot(s) << " = " << lit(P, x0) << ";\n";
        }
        for (int s = n; s < k; ++s) o << "        x[" << s << "] = 0;\n";
        // the warp visits the union of its lanes' columns; each lane adds a column with weight 0 or 1
        o << "        unsigned long long U = warp_or64(G);\n";
        o << "        while (U) {\n            const int p = ctz64(U);\n            U &= U - 1;\n";
        o << "            flip_dyn(p, x, (int)((G >> p) & 1ull));\n        }\n    }\n";
        if (P.dual) {
            emit_dual(B);
            o << "};\n}  // namespace pk\n\n";
            emit_kernel(B);
            return o.str();
        }
        // high chain levels
        auto above = [&](int g) -> std::string {   // the nonempty level just above g
            for (int h = g + 1; h < n; ++h)
                if (P.L.group_begin[h + 1] > P.L.group_begin[h] && h >= B) return "Q" + std::to_string(h);
            return "A::one()";
        };
        if (P.pure_reg) {   // no chain: every step multiplies all rows
            o << "    __device__ __forceinline__ P chain_init(const X (&x)[NX]) { return A::one(); }\n";
            o << "    __device__ __forceinline__ P chain_hi(int j, const X (&x)[NX]) { return A::one(); }\n";
            o << "};\n}  // namespace pk\n\n";
            emit_kernel(B);
            return o.str();
        }
        o << "    __device__ __forceinline__ P chain_init(const X (&x)[NX]) {\n";
        o << "        P q = A::one();\n";
        for (int g : hi) {
            group_product(g, "        ");
            o << "        Q" << g << " = q;\n";
        }
        o << "        return q;\n    }\n";
        // After a flip of column j >= B: rebuild levels j, j-1, ..., B.  The
        // first switch loads the stored level just above j; the second falls
        // through from case j down to case B, so every level's code appears
        // once (the source and the compile time stay linear in n).
        o << "    __device__ __forceinline__ P chain_hi(int j, const X (&x)[NX]) {\n";
        o << "        P q;\n        switch (j) {\n";
        for (int j = B; j < n - 1; ++j) o << "        case " << j << ": q = " << above(j) << "; break;\n";
        o << "        default: q = A::one(); break;\n        }\n";
        o << "        switch (j) {\n";
        for (int j = n - 2; j >= B; --j) {
            o << "        case " << j << ":\n";
            if (P.L.group_begin[j + 1] > P.L.group_begin[j]) {
                group_product(j, "            ");
                o << "            Q" << j << " = q;\n";
            }
            o << "            [[fallthrough]];\n";
        }
        o << "        default: break;\n        }\n";
        o << "        return q;\n    }\n";
        o << "};\n}  // namespace pk\n\n";
        emit_kernel(B);
        return o.str();
    }
    void emit_kernel(int B) {
        o << "extern \"C\" __global__ void __launch_bounds__(" << kCodegenBlock << ", " << min_blocks
          << ") perm_walk(pk::WalkArgs wa, void *xg_base) {\n";
        o << "    extern __shared__ __align__(16) unsigned char perm_xs[];\n";
        o << "    pk::GenPol pol;\n";
        o << "    pol.xs = reinterpret_cast<pk::GenPol::X *>(perm_xs) + threadIdx.x;\n";
        o << "    const unsigned long long tid = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;\n";
        o << "    pol.stride = (unsigned long long)gridDim.x * blockDim.x;\n";
        o << "    pol.xg = reinterpret_cast<pk::GenPol::X *>(xg_base) + tid;\n";
        o << "    pk::walk_tasks<pk::GenPol, pk::A, " << B << ">(pol, wa);\n}\n";
    }
};

// ------------------------------------------------------------------ cache
struct CacheEntry {
    CUmodule module = nullptr;
    CUfunction function = nullptr;
    int regs = 0;
    int local_bytes = 0;   // per-thread local memory (register spills)
    int blocks_per_sm = 0;
};

// A kernel compiled for two resident blocks (128 registers) whose spill
// frame exceeds this is rebuilt for one block (255 registers).  Dense exact
// walks (every row in the lowest group, multi-limb products unrolled over the
// block) are the ones that reach it.
//
// The 128-bit walk of -J_15 with one ring product per row (1.4 KB of spills at
// 128 registers) returns a wrong top limb from that build, reproducibly and for
// every chunk length, while the same source built for 80 or 255 registers is
// right, and the same source compiled as host C++ under address and
// undefined-behaviour sanitizers (with automatic variables initialised to zero
// and to a pattern) matches the CPU oracle chunk by chunk.  The source has no
// defect those checks can see; the wrong result comes from the device build.
// So an exact kernel whose 128-register build spills at all (a frame of any
// size) is also built for 255 registers, both walk the same probe chunks on the
// GPU, and the 128-register build is kept only if the two agree bit for bit.
constexpr int kMaxLocalFrame = 512;

std::mutex g_cache_mu;
std::unordered_map<std::string, CacheEntry> g_cache;
constexpr size_t kCacheMax = 512;

}  // namespace

bool codegen_no_fold() { return no_fold_env(); }

int codegen_block_log2(const perm_plan_s &P) {
    if (P.arith == 0) return P.zero_heavy ? kCodegenBlockLog2ZeroHeavy : kCodegenBlockLog2F64;
    return P.zero_frac > 0.95 && !P.zero_spans ? kCodegenBlockLog2ZeroBlocks : kCodegenBlockLog2Exact;
}

std::string codegen_source(const perm_plan_s &P) {
    Emitter e(P, codegen_min_blocks(P));
    return e.emit();
}

namespace {

// Compiles src with NVRTC for sm_103a and loads it into ce.
perm_status_t compile_and_load(const std::string &src, CacheEntry &ce, std::string &err, size_t smem) {
    Driver &d = driver();
    if (debug_fail(kSiteNvrtc)) { err = "NVRTC compile failed (injected by perm_debug_inject_failures)"; return PERM_ERR_NVRTC; }
    nvrtcProgram prog;
    const char *hdr_src[2] = {perm_embedded_core_cuh, perm_embedded_devmat_h};
    const char *hdr_name[2] = {"core.cuh", "devmat.h"};
    nvrtcResult r = nvrtcCreateProgram(&prog, src.c_str(), "perm_walk.cu", 2, hdr_src, hdr_name);
    if (r != NVRTC_SUCCESS) { err = std::string("nvrtcCreateProgram: ") + nvrtcGetErrorString(r); return PERM_ERR_NVRTC; }
    const char *opts[] = {"--gpu-architecture=sm_103a", "-std=c++17", "-lineinfo", "--device-as-default-execution-space"};
    r = nvrtcCompileProgram(prog, 4, opts);
    if (r != NVRTC_SUCCESS) {
        size_t ls = 0;
        nvrtcGetProgramLogSize(prog, &ls);
        std::string log(ls, '\0');
        if (ls) nvrtcGetProgramLog(prog, &log[0]);
        nvrtcDestroyProgram(&prog);
        err = "NVRTC compile failed: " + log.substr(0, 2000);
        return PERM_ERR_NVRTC;
    }
    size_t cs = 0;
    nvrtcGetCUBINSize(prog, &cs);
    std::vector<char> cubin(cs);
    nvrtcGetCUBIN(prog, cubin.data());
    nvrtcDestroyProgram(&prog);
    cudaFree(nullptr);   // make the primary context current on this thread
    CUresult cr = d.moduleLoadData(&ce.module, cubin.data());
    if (cr != CUDA_SUCCESS) { ce.module = nullptr; err = "cuModuleLoadData: " + cu_err(cr); return PERM_ERR_CUDA; }
    // a loaded module that fails a later step is unloaded, not leaked
    auto unload_fail = [&](const char *what) {
        err = std::string(what) + ": " + cu_err(cr);
        if (d.moduleUnload) d.moduleUnload(ce.module);
        ce = CacheEntry();
        return PERM_ERR_CUDA;
    };
    cr = d.moduleGetFunction(&ce.function, ce.module, "perm_walk");
    if (cr != CUDA_SUCCESS) return unload_fail("cuModuleGetFunction");
    d.funcGetAttribute(&ce.regs, CU_FUNC_ATTRIBUTE_NUM_REGS, ce.function);
    d.funcGetAttribute(&ce.local_bytes, CU_FUNC_ATTRIBUTE_LOCAL_SIZE_BYTES, ce.function);
    if (smem > 48 * 1024) {
        cr = d.funcSetAttribute(ce.function, CU_FUNC_ATTRIBUTE_MAX_DYNAMIC_SHARED_SIZE_BYTES, (int)smem);
        if (cr != CUDA_SUCCESS) return unload_fail("cuFuncSetAttribute");
    }
    cr = d.occupancy(&ce.blocks_per_sm, ce.function, kCodegenBlock, smem);
    if (cr != CUDA_SUCCESS) return unload_fail("occupancy");
    return PERM_OK;
}

}  // namespace

namespace {

// Walks the first chunks of the Gray range (up to 64 warp tasks of 32 chunks
// of 2^K indices) with two builds of the same exact kernel and compares their
// per-task partial sums bit for bit.  Uses its own small device buffers and
// stream.
perm_status_t same_on_probe(const perm_plan_s &P, const CacheEntry &a, const CacheEntry &b, bool *same,
                            std::string &err) {
    Driver &d = driver();
    const int n = P.m.n;
    const int K = std::min(n - 1, codegen_block_log2(P) + 3);
    const uint64_t chunks = std::min<uint64_t>(P.total >> K, 64 * 32);
    const uint64_t ntasks = (chunks + 31) / 32;
    const int words = P.arith;
    const int grid = (int)std::max<uint64_t>(1, (ntasks + 7) / 8);
    const size_t ws_words = 16 + ntasks * (size_t)words;
    const size_t xg_bytes = (size_t)std::max(0, n - P.k - P.k2) * grid * kCodegenBlock * sizeof(int) + 16;
    unsigned char *buf = nullptr;
    cudaStream_t st = nullptr;
    cudaError_t e = cudaMalloc(&buf, 2 * ws_words * 8 + xg_bytes);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    std::vector<uint64_t> out[2];
    const CacheEntry *k[2] = {&a, &b};
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
        uint64_t *ws = reinterpret_cast<uint64_t *>(buf) + i * ws_words;
        e = cudaMemsetAsync(ws, 0, 16 * 8, st);
        if (e != cudaSuccess) break;
        pk::WalkArgs wa;
        wa.chunk_lo = 0;
        wa.chunk_hi = chunks;
        wa.ntasks = ntasks;
        wa.task_counter = reinterpret_cast<unsigned long long *>(ws);
        wa.task_out = reinterpret_cast<unsigned long long *>(ws + 16);
        wa.skip_counter = reinterpret_cast<unsigned long long *>(ws + 1);
        wa.K = K;
        wa.zero_skip = 1;
        wa.timeout_ns = 0;
        wa.deadline_word = reinterpret_cast<unsigned long long *>(ws + 5);
        wa.abort_flag = reinterpret_cast<unsigned int *>(ws + 6);
        void *xg = buf + 2 * ws_words * 8;
        void *params[] = {&wa, &xg};
        if (d.launchKernel(reinterpret_cast<CUfunction>(k[i]->function), (unsigned)grid, 1, 1, kCodegenBlock, 1, 1,
                           (unsigned)P.xs_bytes(), reinterpret_cast<CUstream>(st), params, nullptr) != CUDA_SUCCESS) {
            e = cudaErrorLaunchFailure;
            break;
        }
        out[i].resize(ntasks * (size_t)words);
        e = cudaMemcpyAsync(out[i].data(), ws + 16, out[i].size() * 8, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    if (st) cudaStreamDestroy(st);
    if (buf) cudaFree(buf);
    if (e != cudaSuccess) {
        err = std::string("cross-check of two kernel builds: ") + cudaGetErrorString(e);
        return PERM_ERR_CUDA;
    }
    *same = out[0] == out[1];
    return PERM_OK;
}

}  // namespace

perm_status_t codegen_build(perm_plan_s &P, std::string &err) {
    Driver &d = driver();
    if (!d.ok) { err = "CUDA driver entry points unavailable"; return PERM_ERR_CUDA; }
    const std::string src = codegen_source(P);
    P.cg.block = kCodegenBlock;
    P.cg.block_log2 = codegen_block_log2(P);
    const bool use_cache = !(P.opts.flags & PERM_FLAG_NO_KERNEL_CACHE);
    // a module belongs to one device's context: the cache key names the device
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); dev = -1; }
    const std::string key = "device " + std::to_string(dev) + "\n" + src;
    if (use_cache) {
        std::lock_guard<std::mutex> lk(g_cache_mu);
        auto it = g_cache.find(key);
        if (it != g_cache.end()) {
            P.cg.module = it->second.module;
            P.cg.function = it->second.function;
            P.cg.regs = it->second.regs;
            P.cg.blocks_per_sm = it->second.blocks_per_sm;
            P.cg.cached = true;
            P.regs = P.cg.regs;
            P.ms_compile = 0.0;
            return PERM_OK;
        }
    }
    const double t0 = now_ms();
    CacheEntry ce;
    perm_status_t st = compile_and_load(src, ce, err, P.xs_bytes());
    if (st != PERM_OK) return st;
    const bool fixed_budget = std::getenv("PERM_CODEGEN_MIN_BLOCKS") != nullptr;
    if (ce.local_bytes > kMaxLocalFrame && !fixed_budget && codegen_min_blocks(P) > 1) {
        if (driver().moduleUnload) driver().moduleUnload(ce.module);
        ce = CacheEntry();
        Emitter e1(P, 1);
        st = compile_and_load(e1.emit(), ce, err, P.xs_bytes());
        if (st != PERM_OK) return st;
    } else if (P.arith != 0 && ce.local_bytes > 0 && !fixed_budget) {
        // exact kernel with any spills: cross-check against the 255-register build
        CacheEntry wide;
        Emitter e1(P, 1);
        st = compile_and_load(e1.emit(), wide, err, P.xs_bytes());
        if (st != PERM_OK) { driver().moduleUnload(ce.module); return st; }
        bool same = false;
        st = same_on_probe(P, ce, wide, &same, err);
        if (st != PERM_OK) { driver().moduleUnload(ce.module); driver().moduleUnload(wide.module); return st; }
        if (same) {
            driver().moduleUnload(wide.module);
        } else {
            driver().moduleUnload(ce.module);
            ce = wide;
        }
    }
    P.ms_compile = now_ms() - t0;
    if (use_cache) {
        std::lock_guard<std::mutex> lk(g_cache_mu);
        // another thread may have cached the same kernel meanwhile: this
        // module then stays with the plan
        if (g_cache.size() >= kCacheMax || !g_cache.emplace(key, ce).second) P.cg.owned = true;
    } else {
        P.cg.owned = true;
    }
    P.cg.module = ce.module;
    P.cg.function = ce.function;
    P.cg.regs = ce.regs;
    P.cg.blocks_per_sm = ce.blocks_per_sm;
    P.cg.cached = false;
    P.regs = ce.regs;
    return PERM_OK;
}

cudaError_t codegen_launch(perm_plan_s &P, const pk::WalkArgs &wa, cudaStream_t st) {
    Driver &d = driver();
    pk::WalkArgs a = wa;
    void *xg = P.d_xglob;
    void *params[] = {&a, &xg};
    CUresult r = d.launchKernel(reinterpret_cast<CUfunction>(P.cg.function), (unsigned)P.grid, 1, 1,
                                (unsigned)P.block, 1, 1, (unsigned)P.xs_bytes(), reinterpret_cast<CUstream>(st), params,
                                nullptr);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorLaunchFailure;
}

void codegen_release(perm_plan_s &P) {
    // cached modules live as long as the process; uncached ones go with the plan
    if (P.cg.owned && P.cg.module && driver().moduleUnload)
        driver().moduleUnload(reinterpret_cast<CUmodule>(P.cg.module));
    P.cg.module = nullptr;
    P.cg.function = nullptr;
}

}  // namespace perm
