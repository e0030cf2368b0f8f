// tune.cpp -- autotuned chunk length for the batch walk.
//
// The chunk length K trades start-vector cost (one start vector per 2^K
// steps) and the unrolled-block efficiency against load balance at the tail
// of a persistent launch.  The first batch of each (NMAX, arithmetic) family
// that is large enough times its own group at a few candidate K on a sample of
// its matrices and keeps the fastest; later batches reuse the choice.
#include <map>
#include <mutex>

#include "batch.hpp"

namespace perm {

namespace {
std::mutex g_mu;
std::map<std::pair<int, int>, int> g_choice;
}  // namespace

int tuned_chunk_log2(int nmax, int arith) {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_choice.find({nmax, arith});
    if (it != g_choice.end()) return it->second;
    return 14;
}

void set_tuned_chunk_log2(int nmax, int arith, int K) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_choice[{nmax, arith}] = K;
}

}  // namespace perm
