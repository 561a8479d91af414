// Binomial checkpointing schedule (Sec. 3, Eq. "eqn:recompute").
#pragma once

#include <vector>

namespace ckfwi {

enum { ACT_ADVANCE = 0, ACT_TAKESHOT = 1, ACT_RESTORE = 2, ACT_YOUTURN = 3 };

struct Action {
    int op;   // ACT_*
    int a;    // state (advance: start state)
    int b;    // advance: steps; takeshot / restore: slot
};

// p(n, m): minimal forward steps to reverse n steps with m slots.
long long revolve_p(long long n, long long m);

// Full action list for (N, M); counts = {p, W, R}.  Returns 0 or -1.
int revolve_schedule(int N, int M, std::vector<Action>& acts, long long counts[3]);

// Two storage levels: slots 1 .. H in host memory, H + 1 .. M - 1 on the
// device.  Host checkpoints are taken only in the first forward sweep, at
// the starts of segments; each segment is then reversed (last first) from
// its start by Revolve in the device slots (multistage checkpointing, the
// scheme of Stumm and Walther the paper builds its model on).  The segments
// minimise the forward steps within that family.  Returns 0 or -1.
int multistage_schedule(int N, int M, int H, std::vector<Action>& acts, long long counts[3]);

}  // namespace ckfwi
