// round_order.h -- the claim order of a refactorization round's columns (host).
//
// A round processes, for each active task, its columns from the task's start
// column to its end.  The warps claim them in the order given here: ascending
// within a task (a column's steps in its own task come before it, so a column
// never waits for one that is not yet claimed, and the earliest unfinished
// claimed column can always proceed), the tasks interleaved in proportion to
// their lengths, so that every task advances through its columns at the same
// rate.  Claimed task by task instead, the columns near the top of the first
// tasks' elimination trees hold the resident warps while they wait for their
// chains, and the later tasks start late.
#pragma once

#include <cstdint>
#include <utility>
#include <vector>

namespace bk {

// ranges[k] = [lo, hi): the columns of the k-th active task.  Column i of a task
// of L columns goes to bucket floor((2i + 1) N / 2L) of N buckets (N columns in
// all), which grows strictly with i (N >= L); a counting sort over the buckets
// keeps each task's order and, within a bucket, the tasks' order.
inline void bk_round_order(const std::vector<std::pair<int32_t, int32_t>> &ranges, std::vector<int32_t> &cols)
{
    int64_t N = 0;
    for (const auto &r : ranges) N += r.second > r.first ? r.second - r.first : 0;
    cols.assign((size_t)N, 0);
    if (N == 0) return;
    std::vector<int64_t> at((size_t)N + 1, 0);
    auto bucket = [N](int64_t i, int64_t L) { return (size_t)(((2 * i + 1) * N) / (2 * L)); };
    for (const auto &r : ranges) {
        const int64_t L = r.second - r.first;
        for (int64_t i = 0; i < L; i++) at[bucket(i, L) + 1]++;
    }
    for (size_t b = 0; b < (size_t)N; b++) at[b + 1] += at[b];
    for (const auto &r : ranges) {
        const int64_t L = r.second - r.first;
        for (int64_t i = 0; i < L; i++) cols[(size_t)at[bucket(i, L)]++] = r.first + (int32_t)i;
    }
}

}  // namespace bk
