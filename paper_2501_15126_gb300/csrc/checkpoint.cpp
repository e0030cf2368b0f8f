// checkpoint.cpp -- resumable runs over Gray-index slices.
//
// A permanent's walk splits into independent aligned ranges of Gray indices
// (Sec. II-A): the partial sums of any partition add up to the whole.  A run
// therefore checkpoints by recording each finished slice's partial sum in a
// small text file; a run that stopped (killed, timed out, machine lost)
// resumes by skipping the recorded slices.  Slices are combined in slice
// order -- compensated FP64 additions, or wrapping ring additions on the exact
// path -- so the result is the same bits however the run was split across
// calls.
#include <cinttypes>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "plan.hpp"

namespace perm {

namespace {

void fnv_mix(uint64_t &h, const void *p, size_t nb) {
    const unsigned char *c = static_cast<const unsigned char *>(p);
    for (size_t i = 0; i < nb; ++i) { h ^= c[i]; h *= 1099511628211ull; }
}

// FNV-1a over everything that determines the walk: n, arithmetic, order and values.
uint64_t walk_hash(const perm_plan_s &P) {
    uint64_t h = 14695981039346656037ull;
    const int n = P.m.n;
    const int dd = P.dd ? 1 : 0;
    fnv_mix(h, &n, sizeof n);
    fnv_mix(h, &P.arith, sizeof P.arith);
    fnv_mix(h, &dd, sizeof dd);
    fnv_mix(h, P.L.col_order, sizeof(int) * n);
    const size_t nb = (size_t)n * n * 8;
    fnv_mix(h, P.m.is_int ? (const void *)P.m.v : (const void *)P.m.f, nb);
    return h;
}

// Check word of one slice record: FNV-1a over its index and words.
uint64_t slice_check(uint64_t idx, const uint64_t *w, int words) {
    uint64_t h = 14695981039346656037ull;
    fnv_mix(h, &idx, sizeof idx);
    fnv_mix(h, w, sizeof(uint64_t) * words);
    return h;
}

bool parse_hex16(const char *t, size_t len, uint64_t *out) {
    if (len != 16) return false;
    uint64_t v = 0;
    for (size_t i = 0; i < 16; ++i) {
        const char c = t[i];
        int d;
        if (c >= '0' && c <= '9') d = c - '0';
        else if (c >= 'a' && c <= 'f') d = c - 'a' + 10;
        else return false;
        v = (v << 4) | (uint64_t)d;
    }
    *out = v;
    return true;
}

// One slice record: "slice <index> <word> ... <check>\n" with `words` words
// and the check word of exactly 16 lower-case hex digits each.  A torn,
// joined or altered line (a run stopped mid-write) fails and is recomputed.
bool parse_slice(const char *line, int words, uint64_t nslices, uint64_t *idx, uint64_t *w) {
    const size_t len = std::strlen(line);
    if (len < 7 || line[len - 1] != '\n' || std::strncmp(line, "slice ", 6) != 0) return false;
    const char *p = line + 6;
    uint64_t v = 0;
    int digits = 0;
    while (*p >= '0' && *p <= '9' && digits < 20) { v = v * 10 + (uint64_t)(*p - '0'); ++p; ++digits; }
    if (!digits || *p != ' ' || v >= nslices) return false;
    *idx = v;
    uint64_t check = 0;
    for (int k = 0; k <= words; ++k) {
        if (*p != ' ') return false;
        ++p;
        const char *t = p;
        while (*p && *p != ' ' && *p != '\n') ++p;
        if (!parse_hex16(t, (size_t)(p - t), k < words ? &w[k] : &check)) return false;
    }
    if (*p != '\n' || p[1] != 0) return false;
    return check == slice_check(*idx, w, words);
}

void two_sum(double a, double b, double *s, double *e) {
    *s = a + b;
    const double bb = *s - a;
    *e = (a - (*s - bb)) + (b - bb);
}

}  // namespace

}  // namespace perm

using namespace perm;

extern "C" perm_status_t perm_checkpoint_run(const perm_matrix_t *A, const perm_opts_t *opts_in, const char *path,
                                             int32_t slice_log2, int32_t max_slices, void *stream,
                                             perm_result_t *out) {
    if (!A || !path || !out) return fail(PERM_ERR_ARG, "NULL argument");
    std::memset(out, 0, sizeof(*out));
    perm_opts_t opts;
    std::memset(&opts, 0, sizeof(opts));
    if (opts_in) opts = *opts_in;
    if (opts.g_lo || opts.g_hi) return fail(PERM_ERR_ARG, "a checkpointed run covers the whole range");
    perm_plan_s whole;
    perm_status_t st = plan_prepare(A, &opts, whole);
    if (st != PERM_OK) return st;
    const int n = whole.m.n;
    if (slice_log2 < 5 || slice_log2 > n - 1) return fail(PERM_ERR_ARG, "slice_log2 must be in [5, n-1]");
    if (max_slices < 0) return fail(PERM_ERR_ARG, "max_slices < 0");
    describe(whole, out);
    if (whole.zero) { out->status = PERM_OK; return PERM_OK; }
    const uint64_t slice = 1ull << slice_log2;
    const uint64_t nslices = whole.total / slice;
    const uint64_t hash = walk_hash(whole);
    const int words = result_words(whole.arith);   // FP64: hi, lo, sum|terms|

    // read what is already recorded
    std::map<uint64_t, std::vector<uint64_t>> done;
    bool header_ok = false, ends_in_newline = true;
    if (FILE *f = std::fopen(path, "r")) {
        char line[512];
        while (std::fgets(line, sizeof line, f)) {
            const size_t len = std::strlen(line);
            ends_in_newline = len > 0 && line[len - 1] == '\n';
            uint64_t fh = 0;
            int fn = 0, fa = 0, fk = 0, fd = 0;
            if (std::sscanf(line, "perm-checkpoint v2 hash=%" SCNx64 " n=%d arith=%d dd=%d slice_log2=%d", &fh, &fn,
                            &fa, &fd, &fk) == 5) {
                if (fh != hash || fn != n || fa != whole.arith || fd != (whole.dd ? 1 : 0) || fk != slice_log2) {
                    std::fclose(f);
                    return fail(PERM_ERR_ARG, "checkpoint file belongs to another matrix, order, arithmetic or slice size");
                }
                header_ok = true;
                continue;
            }
            uint64_t idx = 0, w[3] = {0, 0, 0};
            if (header_ok && parse_slice(line, words, nslices, &idx, w)) done[idx] = std::vector<uint64_t>(w, w + words);
        }
        std::fclose(f);
    }
    FILE *f = std::fopen(path, "a");
    if (!f) return fail(PERM_ERR_ARG, "cannot open the checkpoint file for appending");
    if (!ends_in_newline) std::fputc('\n', f);   // never glue a record onto a torn line
    if (!header_ok) {
        std::fprintf(f, "perm-checkpoint v2 hash=%016" PRIx64 " n=%d arith=%d dd=%d slice_log2=%d\n", hash, n,
                     whole.arith, whole.dd ? 1 : 0, slice_log2);
        std::fflush(f);
    }

    // compute missing slices
    int32_t computed = 0;
    double ms_kernel = 0.0, ms_compile = 0.0;
    for (uint64_t i = 0; i < nslices; ++i) {
        if (done.count(i)) continue;
        if (max_slices && computed >= max_slices) break;
        perm_opts_t so = opts;
        so.g_lo = i * slice;
        so.g_hi = (i + 1) * slice;
        perm_plan_t p = nullptr;
        st = perm_plan_create(A, &so, &p);
        if (st != PERM_OK) { std::fclose(f); return st; }
        perm_result_t r;
        st = perm_compute(p, stream, &r);
        perm_plan_destroy(p);
        if (st != PERM_OK) { std::fclose(f); return st; }
        std::vector<uint64_t> w(words);
        if (whole.arith == 0) {
            std::memcpy(&w[0], &r.f64, 8);
            std::memcpy(&w[1], &r.f64_lo, 8);
            std::memcpy(&w[2], &r.abs_term_sum, 8);
        } else {
            for (int k = 0; k < words; ++k) w[k] = r.partial[k];
        }
        std::fprintf(f, "slice %" PRIu64, i);
        for (int k = 0; k < words; ++k) std::fprintf(f, " %016" PRIx64, w[k]);
        std::fprintf(f, " %016" PRIx64 "\n", slice_check(i, w.data(), words));
        std::fflush(f);
        done[i] = w;
        ++computed;
        ms_kernel += r.ms_kernel;
        ms_compile += r.ms_compile;
    }
    std::fclose(f);
    out->steps = (uint64_t)done.size() * slice;
    out->ms_kernel = ms_kernel;
    out->ms_compile = ms_compile;
    if (done.size() < nslices) {
        out->status = PERM_ERR_NOT_READY;
        return PERM_ERR_NOT_READY;
    }
    // combine in slice order
    uint64_t raw[3] = {0, 0, 0};
    if (whole.arith == 0) {
        double hi = 0.0, lo = 0.0, ab = 0.0;
        for (auto &kv : done) {
            double a, b, c, s, e;
            std::memcpy(&a, &kv.second[0], 8);
            std::memcpy(&b, &kv.second[1], 8);
            std::memcpy(&c, &kv.second[2], 8);
            two_sum(hi, a, &s, &e);
            hi = s;
            lo += e + b;
            ab += c;
        }
        double s, e;
        two_sum(hi, lo, &s, &e);
        std::memcpy(&raw[0], &s, 8);
        std::memcpy(&raw[1], &e, 8);
        // finish_raw scales the third word by 2^abs_shift: hand it the unscaled sum
        ab = std::ldexp(ab, -whole.abs_shift);
        std::memcpy(&raw[2], &ab, 8);
    } else {
        for (auto &kv : done) {
            unsigned carry = 0;
            for (int k = 0; k < words; ++k) {
                const unsigned __int128 t = (unsigned __int128)raw[k] + kv.second[k] + carry;
                raw[k] = (uint64_t)t;
                carry = (unsigned)(t >> 64);
            }
        }
    }
    st = finish_raw(whole, raw, out);
    out->steps = whole.total;
    out->ms_kernel = ms_kernel;
    out->ms_compile = ms_compile;
    return st;
}
