// Binomial checkpointing schedule (Sec. 3, Eq. "eqn:recompute").
//
// p(N, M), the minimal number of forward steps to reverse N steps with M
// checkpoint slots (the initial state's slot included), is evaluated with
// Griewank's closed form: with beta(s, r) = C(s + r, s) and r the smallest
// integer such that beta(M, r) >= N,  p = r N - C(M + r, M + 1).
// The schedule splits a range of n steps with m slots at the smallest
// Nt in [1, n-1] minimising Nt + p(Nt, m) + p(n - Nt, m - 1) (the paper's
// recursion; its upper limit N is read as N - 1, since Nt = N would refer to
// p(N, M) itself), stores the state at the split in the next slot, reverses
// the right part with one slot fewer, restores and reverses the left part.
// With one slot left the range is reversed by re-advancing from its start.
#include "revolve.h"

#include <algorithm>
#include <vector>

namespace ckfwi {

long long revolve_p(long long n, long long m)
{
    if (n <= 1) return 0;
    if (m >= n) return n - 1;
    if (m == 1) return n * (n - 1) / 2;
    // beta = C(m + r, m), grown until it reaches n
    long long r = 0, beta = 1;
    while (beta < n) {
        ++r;
        beta = beta * (m + r) / r;
    }
    // C(m + r, m + 1) = C(m + r, r - 1) = beta * r / (m + 1)
    const long long c = beta * r / (m + 1);
    return r * n - c;
}

namespace {

struct Builder {
    std::vector<std::vector<long long>> tab;   // tab[m][n] = p(n, m)
    std::vector<Action>* out;
    long long p = 0, W = 0, R = 0;
    // slot numbers as emitted: the range's own start slot 0 is `start`,
    // slot i >= 1 is dev0 + i
    long long start = 0, dev0 = 0;

    long long P(long long n, long long m) const { return tab[m][n]; }

    void emit(int op, long long a, long long b)
    {
        if (op == ACT_TAKESHOT || op == ACT_RESTORE) b = b == 0 ? start : dev0 + b;
        out->push_back(Action{op, (int)a, (int)b});
        if (op == ACT_ADVANCE) p += b;
        if (op == ACT_TAKESHOT) ++W;
        if (op == ACT_RESTORE) ++R;
    }

    long long split(long long n, long long m) const
    {
        long long best = 1, cost = -1;
        for (long long t = 1; t <= n - 1; ++t) {
            const long long c = t + P(t, m) + P(n - t, m - 1);
            if (cost < 0 || c < cost) {
                cost = c;
                best = t;
            }
        }
        return best;
    }

    // state s is current and held in `slot`
    void rev(long long s, long long n, long long m, long long slot)
    {
        while (true) {
            if (n == 1) {
                emit(ACT_YOUTURN, s, 0);
                return;
            }
            if (m == 1) {
                for (long long j = n - 1; j >= 1; --j) {
                    if (j != n - 1) emit(ACT_RESTORE, s, slot);
                    emit(ACT_ADVANCE, s, j);
                    emit(ACT_YOUTURN, s + j, 0);
                }
                emit(ACT_RESTORE, s, slot);
                emit(ACT_YOUTURN, s, 0);
                return;
            }
            const long long t = split(n, m);
            emit(ACT_ADVANCE, s, t);
            emit(ACT_TAKESHOT, s + t, slot + 1);
            rev(s + t, n - t, m - 1, slot + 1);
            emit(ACT_RESTORE, s, slot);
            n = t;          // tail call: rev(s, t, m, slot)
        }
    }
};

}  // namespace

int revolve_schedule(int N, int M, std::vector<Action>& acts, long long counts[3])
{
    if (N < 1 || M < 1) return -1;
    const long long mm = std::min<long long>(M, N);
    Builder B;
    B.out = &acts;
    B.tab.assign(mm + 1, std::vector<long long>(N + 1, 0));
    for (long long m = 1; m <= mm; ++m)
        for (long long n = 0; n <= N; ++n) B.tab[m][n] = revolve_p(n, m);
    acts.clear();
    B.rev(0, N, mm, 0);
    if (counts) {
        counts[0] = B.p;
        counts[1] = B.W;
        counts[2] = B.R;
    }
    return 0;
}

int multistage_schedule(int N, int M, int H, std::vector<Action>& acts, long long counts[3])
{
    if (N < 1 || M < 1 || H < 0 || H > M - 1) return -1;
    const long long md = M - H;                        // a segment's start plus the device slots
    std::vector<long long> pd(N + 1);
    for (long long n = 0; n <= N; ++n) pd[n] = revolve_p(n, md);
    // k segments of the first sweep (equal lengths: p is convex in n, so an
    // even split minimises their sum) and a last segment of L steps, which
    // the first sweep does not cross
    auto cost = [&](long long k, long long L) {
        long long c = (N - L) + pd[L];
        if (k > 0) {
            const long long q = (N - L) / k, rem = (N - L) % k;
            c += rem * pd[q + 1] + (k - rem) * pd[q];
        }
        return c;
    };
    long long bk = 0, bL = N, best = pd[N];
    for (long long k = 1; k <= std::min<long long>(H, N - 1); ++k)
        for (long long L = 1; L <= N - k; ++L) {
            const long long c = cost(k, L);
            if (c < best) {
                best = c;
                bk = k;
                bL = L;
            }
        }
    std::vector<long long> b0(bk + 2, 0), len(bk + 1, 0);
    if (bk > 0) {
        const long long q = (N - bL) / bk, rem = (N - bL) % bk;
        for (long long j = 0; j < bk; ++j) len[j] = q + (j < rem ? 1 : 0);
    }
    len[bk] = bL;
    for (long long j = 0; j <= bk; ++j) b0[j + 1] = b0[j] + len[j];
    Builder B;
    B.out = &acts;
    const long long mm = std::min<long long>(md, N);
    B.tab.assign(mm + 1, std::vector<long long>(N + 1, 0));
    for (long long m = 1; m <= mm; ++m)
        for (long long n = 0; n <= N; ++n) B.tab[m][n] = revolve_p(n, m);
    acts.clear();
    B.dev0 = H;
    // first sweep: host slot j holds the start of segment j (j = 1 .. k)
    for (long long j = 1; j <= bk; ++j) {
        B.start = 0;
        B.out->push_back(Action{ACT_ADVANCE, (int)b0[j - 1], (int)len[j - 1]});
        B.p += len[j - 1];
        B.out->push_back(Action{ACT_TAKESHOT, (int)b0[j], (int)j});
        ++B.W;
    }
    // reversal, last segment first; its start slot is the segment's host slot
    for (long long j = bk; j >= 0; --j) {
        B.start = j;
        if (j < bk) {
            B.out->push_back(Action{ACT_RESTORE, (int)b0[j], (int)j});
            ++B.R;
        }
        B.rev(b0[j], len[j], std::min(md, len[j]), 0);
    }
    if (counts) {
        counts[0] = B.p;
        counts[1] = B.W;
        counts[2] = B.R;
    }
    return 0;
}

}  // namespace ckfwi
