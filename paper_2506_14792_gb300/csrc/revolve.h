// Binomial checkpointing schedule for the reverse sweep (Griewank & Walther's revolve
// family; the paper's timestepper adjoints use the checkpoint_schedules library for the
// same purpose, Supplementary A.4).
//
// With s free slots and t forward repetitions, at most beta(s, t) = C(s + t, s) steps can
// be reversed.  A segment [a, b) whose start state X_a is held in a slot is reversed by
// advancing to a split point m, storing X_m, reversing [m, b) with s - 1 slots, freeing
// the slot and reversing [a, m) with s slots; the split keeps the right part within
// beta(s - 1, t) and the left part within beta(s, t - 1), t minimal for the segment.
// Slot 0 holds the initial state.  Actions are executed in order by the caller.
//
// Two-level variant (plan2): besides the s device slots, h slots in host memory (the paper's
// optimal-dynamo setup II keeps checkpoints in RAM and on disk, Supplementary Table on the
// Taylor-remainder tests; H-revolve of Herrmann & Pallez).  The first forward sweep stores
// X_a on the host at the start of every segment [a, a + K), K = ceil(N / h); the segments are
// then reversed last first, each from its host copy by the binomial schedule on the device
// slots.  Host slots are numbered s .. s + h - 1 in the actions.
#pragma once
#include <algorithm>
#include <vector>

namespace spadj {

enum CkptAction { CK_ADVANCE = 0, CK_STORE = 1, CK_RESTORE = 2, CK_ADJOINT = 3, CK_FREE = 4, CK_OBJECTIVE = 5 };

struct CkptOp {
  int type, a, b, slot;  // ADVANCE: a -> b; STORE/RESTORE/FREE: state a in slot; ADJOINT: step a
};

inline double ck_beta(int s, int t) {  // C(s + t, s), as double to avoid overflow
  double r = 1.0;
  for (int i = 1; i <= s; ++i) r = r * (t + i) / i;
  return r;
}

struct CkptPlanner {
  int n_steps;
  std::vector<CkptOp> ops;
  std::vector<int> free_slots;
  bool objective_done = false;

  int take_slot() {
    int s = free_slots.back();
    free_slots.pop_back();
    return s;
  }

  void rev(int a, int b, int slot_a) {
    const int l = b - a;
    if (l <= 0) return;
    if (l == 1) {
      if (b == n_steps && !objective_done) {
        ops.push_back({CK_RESTORE, a, 0, slot_a});
        ops.push_back({CK_ADVANCE, a, b, -1});
        ops.push_back({CK_OBJECTIVE, b, 0, -1});
        objective_done = true;
      }
      ops.push_back({CK_RESTORE, a, 0, slot_a});
      ops.push_back({CK_ADJOINT, a, 0, -1});
      return;
    }
    const int s = (int)free_slots.size();
    if (s == 0) {  // no slot left: recompute each step from X_a
      for (int k = b - 1; k >= a; --k) {
        if (k + 1 == n_steps && !objective_done) {
          ops.push_back({CK_RESTORE, a, 0, slot_a});
          ops.push_back({CK_ADVANCE, a, n_steps, -1});
          ops.push_back({CK_OBJECTIVE, n_steps, 0, -1});
          objective_done = true;
        }
        ops.push_back({CK_RESTORE, a, 0, slot_a});
        if (k > a) ops.push_back({CK_ADVANCE, a, k, -1});
        ops.push_back({CK_ADJOINT, k, 0, -1});
      }
      return;
    }
    int t = 1;
    while (ck_beta(s, t) < l) ++t;
    double r = ck_beta(s - 1, t);
    int l2 = (r < (double)(l - 1)) ? (int)r : l - 1;
    const int m = b - l2;
    ops.push_back({CK_RESTORE, a, 0, slot_a});
    ops.push_back({CK_ADVANCE, a, m, -1});
    const int sm = take_slot();
    ops.push_back({CK_STORE, m, 0, sm});
    rev(m, b, sm);
    ops.push_back({CK_FREE, m, 0, sm});
    free_slots.push_back(sm);
    rev(a, m, slot_a);
  }

  // total_slots >= 1 (slot 0 = initial state).  with_objective = false: the caller supplies the
  // cotangent of X_steps (a segment of a longer sweep), so no CK_OBJECTIVE is planned.
  std::vector<CkptOp> plan(int steps, int total_slots, bool with_objective = true) {
    n_steps = steps;
    ops.clear();
    free_slots.clear();
    objective_done = !with_objective;
    for (int sl = total_slots - 1; sl >= 1; --sl) free_slots.push_back(sl);
    ops.push_back({CK_STORE, 0, 0, 0});
    rev(0, steps, 0);
    return ops;
  }

  // Two-level schedule with total_slots device slots and host_slots >= 1 host slots.
  std::vector<CkptOp> plan2(int steps, int total_slots, int host_slots) {
    std::vector<CkptOp> out;
    const int K = (steps + host_slots - 1) / host_slots;
    const int nseg = (steps + K - 1) / K;
    for (int j = 0; j < nseg; ++j) {
      if (j > 0) out.push_back({CK_ADVANCE, (j - 1) * K, j * K, -1});
      out.push_back({CK_STORE, j * K, 0, total_slots + j});
    }
    for (int j = nseg - 1; j >= 0; --j) {
      const int a = j * K, b = std::min(steps, a + K);
      out.push_back({CK_RESTORE, a, 0, total_slots + j});
      CkptPlanner sub;
      for (CkptOp o : sub.plan(b - a, std::min(total_slots, b - a + 1), b == steps)) {
        o.a += a;
        if (o.type == CK_ADVANCE) o.b += a;
        out.push_back(o);
      }
      out.push_back({CK_FREE, a, 0, 0});
      out.push_back({CK_FREE, a, 0, total_slots + j});
    }
    return out;
  }
};

}  // namespace spadj
