// devmat.h -- plain-old-data shared by the host code and the kernels (and
// handed to NVRTC as a header of the generated kernels): the launch
// arguments of the walk and the matrix image read by the generic kernels.
// No standard headers, so NVRTC can compile it as is.
#pragma once

namespace pk {

// Launch arguments of one Gray-code walk (see core.cuh).
struct WalkArgs {
    unsigned long long chunk_lo;        // first chunk index (in units of 2^K Gray indices)
    unsigned long long chunk_hi;        // one past the last chunk index
    unsigned long long ntasks;          // ceil((chunk_hi - chunk_lo) / 32): one task = 32 chunks
    unsigned long long *task_counter;   // zeroed before the launch; warps take tasks from it
    unsigned long long *task_out;       // ntasks * words: one warp-reduced result per task
    unsigned long long *skip_counter;   // blocks skipped as all-zero (may be null)
    int K;                              // log2 of the chunk length (>= B)
    int zero_skip;                      // 1 = skip all-zero blocks
    unsigned long long timeout_ns;      // device-side deadline, counted from the first task fetch (0 = none)
    unsigned long long *deadline_word;  // zeroed before the launch; the first warp stores its deadline
    unsigned int *abort_flag;           // set to 1 by a warp that stopped at the deadline
};

// One entry of a generic (multi-matrix) walk: the launch's tasks
// [task_begin, next entry's task_begin) walk chunks chunk_lo + 32 t + lane
// (t counted from task_begin) of the matrix image `image`, and task t's
// result goes to task_out[(out_offset + t - task_begin) * words].  A batch
// has out_offset == task_begin; the serving loop points several launches'
// slices of one request at that request's own result range.
struct BatchMat {
    unsigned long long task_begin;
    unsigned long long chunk_lo;
    unsigned long long chunk_hi;
    unsigned long long out_offset;
    int image;
    int K;
    int abs_shift;                      // FP64 / double-double: sum|terms| is kept as sum|terms| 2^-abs_shift
    int reserved;
};

// Launch arguments of the generic kernels: any number of matrices of one
// NMAX bucket and one arithmetic, their images packed in devmats.
struct BatchArgs {
    const BatchMat *mats;
    const void *devmats;                // images; BatchMat::image is an offset in 16-byte units
    unsigned long long ntasks;          // sum of all matrices' tasks
    unsigned long long *task_counter;   // zeroed before the launch
    unsigned long long *task_out;       // results, indexed through BatchMat::out_offset
    unsigned long long *skip_counter;   // may be null
    unsigned long long slot_bytes;      // per-warp shared-memory slot (>= every image's bytes)
    int nmat;
    int zero_skip;
    unsigned long long timeout_ns;      // device-side deadline, counted from the first task fetch (0 = none)
    unsigned long long *deadline_word;  // zeroed before the launch; the first warp stores its deadline
    unsigned int *abort_flag;           // set to 1 by a warp that stopped at the deadline
};

// The ordered matrix as the generic kernels read it (a variable-length
// image; only the first `bytes` bytes exist).  Slots are rows in the plan's
// order; positions are columns in the plan's order.  Column p's values, in
// slot order, are val[colptr[p] ..].  V is double (FP64 path) or int (exact
// path: values doubled).  Slots are numbered group by group (a row's group is
// the first column position that touches it), so group m is the contiguous
// slot range [gbegin[m], gbegin[m+1]); group 0 is exactly column 0's rows.
// Group 0 is sorted by the next column that touches each of its rows: S_m,
// the rows of column 0 next touched by column m, are the contiguous slots
// [sbegin[m], sbegin[m+1]).  For NMAX in {16, 32, 48} the header is
// 48 + 12 NMAX bytes, a multiple of 16.  X0 is the type of the start values:
// V itself, except on the double-double path, whose start values are exact
// pairs of doubles (hi, lo) while the matrix values stay doubles.
template <int NMAX, typename V, typename X0 = V>
struct DevMat {
    int n;                              // dimension
    int top;                            // highest m with group m or S_m nonempty
    int nnz;                            // values stored (columns 0..n-2)
    int bytes;                          // size of this image, a multiple of 16
    unsigned long long colmask[NMAX];   // slots touched by column position p (p < n-1)
    unsigned short colptr[NMAX];        // first value of column p
    unsigned char gbegin[NMAX + 16];    // first slot of group m (m <= n; gbegin[n] = n)
    unsigned char sbegin[NMAX + 16];    // first slot of S_m (1 <= m <= n; sbegin[n] = |group 0|)
    X0 x0[NMAX];                        // Nijenhuis-Wilf start values by slot
    V val[NMAX * NMAX];                 // nnz values, column after column
};

}  // namespace pk
