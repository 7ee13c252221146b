// Host-side plan of the scheduled sketch product A S (sketch_sched.cu).
//
// The product: column c of A~ = A S is the sum, over the bucket of c (the rows
// j of S whose non-zeros fall in column c, Lemma 3.2 item 2), of
// sign(j, c) A[:, j] / sqrt(s).  The kernel holds one whole row of A in shared
// memory and gives each output column to one lane, which gathers the row
// elements of its bucket.  A warp reads 32 row elements per step; the step is
// one shared-memory wavefront only if the 32 elements sit in 32 different
// banks (bank = j mod 32).  This file decides, once per sketch, which element
// each lane reads at each step:
//
//   1. Columns are split into parts only where a column has more entries than
//      one lane's register budget holds; parts are grouped 32 to a warp.
//   2. Each warp runs a "+" phase and a "-" phase (entries of sign +1, then
//      -1), so the kernel adds or subtracts without reading a sign.  Its step
//      count is T+ + T-, where T+ is the larger of its busiest lane and its
//      busiest bank among the + entries (likewise T-).  A local search swaps
//      parts between warps to lower the sum of the warps' step counts: it
//      evens out the per-bank loads of each warp.
//   3. Each phase of each warp is a bipartite multigraph (32 lanes x 32 banks,
//      one edge per entry).  By Konig's edge-colouring theorem its edges split
//      into exactly (maximum degree) matchings; colour c is step c, so no two
//      lanes meet in a bank.  The colouring is built edge by edge, flipping an
//      alternating two-colour path when the free colours of the two ends
//      differ.
//   4. Lanes without an entry at a step read a zero pad element in a bank that
//      the step leaves free.
//
// Plain C++, no CUDA: the library runs it on the host, and the CPU tests run
// it through spm_sched_plan_host.
#pragma once

#include <stdint.h>

#include <algorithm>
#include <numeric>
#include <vector>

namespace spm {
namespace sched {

#ifndef SCHED_STEPS
#define SCHED_STEPS 96
#endif
static constexpr int kTT = SCHED_STEPS;  // steps per lane per row, both phases (kTT / 2 registers)
static constexpr int kLanes = 1024;   // lanes (threads) per CTA
static constexpr int kWarps = 32;
static constexpr int kPad = 32;       // zero floats ahead of each row, one per bank
static constexpr int kLaneCap = 90;   // a column part holds at most this many entries
static constexpr int kSignCap = 48;   // ... and at most this many of either sign
static constexpr int kStripe = 4;     // warps per stripe of the initial grouping

struct GroupPlan {
  std::vector<uint32_t> words;   // kWarps x (kTT / 2) x 32: two 15-bit row offsets per word, the
                                 // even step's in bits 0-14, the odd step's in bits 17-31
  std::vector<int32_t> wsteps;   // kWarps x 2: steps of the + and the - phase
  std::vector<int32_t> slot;     // kLanes: staging slot of each lane (-1: idle lane), plus
                                 // kLanes << 16 when the lane gathers its part negated
  std::vector<int32_t> partner;  // columns of the group: slot of a column's second part, or -1
  int64_t steps = 0;             // sum over warps of T+ + T-
};

namespace detail {

struct Part {
  int col = 0;                  // column inside the group
  int which = 0;                // 0: first or only part, 1: second part of a split column
  bool neg = false;             // gathered negated: ent[0] holds its - entries, ent[1] its +
  std::vector<uint16_t> ent[2]; // row offsets (kPad + j) gathered in the + and the - phase
  int bank[2][32] = {};         // per-bank entry counts of each phase
};

inline void flip(Part& p) {
  p.neg = !p.neg;
  std::swap(p.ent[0], p.ent[1]);
  for (int b = 0; b < 32; ++b) std::swap(p.bank[0][b], p.bank[1][b]);
}

struct Rng {  // xorshift64: a fixed, portable sequence
  uint64_t x;
  uint32_t next() {
    x ^= x << 13;
    x ^= x >> 7;
    x ^= x << 17;
    return (uint32_t)(x >> 16);
  }
};

struct WarpSet {
  int lane[32];
  int bank[2][32];
};

inline int phase_steps(const std::vector<Part>& parts, const WarpSet& w, int sg) {
  int t = 0;
  for (int k = 0; k < 32; ++k)
    if (w.lane[k] >= 0) t = std::max(t, (int)parts[w.lane[k]].ent[sg].size());
  for (int b = 0; b < 32; ++b) t = std::max(t, w.bank[sg][b]);
  return t;
}

inline int warp_cost(const std::vector<Part>& parts, const WarpSet& w) {
  const int t = phase_steps(parts, w, 0) + phase_steps(parts, w, 1);
  return t + (t > kTT ? 100000 : 0);  // a warp over the register budget is infeasible
}

inline void add_part(const std::vector<Part>& parts, WarpSet& w, int k, int pi, int dir) {
  if (pi < 0) return;
  for (int sg = 0; sg < 2; ++sg)
    for (int b = 0; b < 32; ++b) w.bank[sg][b] += dir * parts[pi].bank[sg][b];
  (void)k;
}

// Proper edge colouring of a bipartite multigraph (32 lanes x 32 banks) with
// D colours, D at least the maximum degree: colour of each edge in col.
inline void colour(const std::vector<int>& eu, const std::vector<int>& ev, int D,
                   std::vector<int>& col) {
  const int E = (int)eu.size();
  std::vector<int> U(32 * D, -1), V(32 * D, -1);  // U[u D + c]: edge of colour c at lane u
  std::vector<int> path;
  col.assign(E, -1);
  for (int e = 0; e < E; ++e) {
    const int u = eu[e], v = ev[e];
    int a = 0;
    while (U[u * D + a] >= 0) ++a;  // free at u (deg u < D before this edge)
    int b = 0;
    while (V[v * D + b] >= 0) ++b;  // free at v
    if (V[v * D + a] >= 0) {
      if (U[u * D + b] < 0) {
        a = b;  // b is free at both ends
      } else {
        // the a/b path from v (v -a- lane -b- bank -a- ...) cannot reach u, which
        // has no a edge; swapping a and b along it frees a at v
        path.clear();
        int x = v, c = a;
        bool at_bank = true;
        for (;;) {
          const int f = at_bank ? V[x * D + c] : U[x * D + c];
          if (f < 0) break;
          path.push_back(f);
          x = at_bank ? eu[f] : ev[f];
          at_bank = !at_bank;
          c = (c == a) ? b : a;
        }
        for (int f : path) {
          U[eu[f] * D + col[f]] = -1;
          V[ev[f] * D + col[f]] = -1;
        }
        for (int f : path) {
          col[f] = (col[f] == a) ? b : a;
          U[eu[f] * D + col[f]] = f;
          V[ev[f] * D + col[f]] = f;
        }
      }
    }
    col[e] = a;
    U[u * D + a] = e;
    V[v * D + a] = e;
  }
}

}  // namespace detail

// Plans one column group.  cols[c] lists the entries of column c of the group
// as j | (sign bit 31 set = minus), j ascending.  search: local-search moves.
// Returns false if the group does not fit the kernel (then nothing is usable).
inline bool plan_group(const std::vector<std::vector<uint32_t>>& cols, int64_t search,
                       GroupPlan& out) {
  using namespace detail;
  const int cw = (int)cols.size();
  if (cw < 1 || cw > kLanes) return false;
  std::vector<Part> parts;
  parts.reserve(kLanes);
  out.partner.assign(cw, -1);
  // 1. parts: a column with more entries than one lane holds must be split in
  // two; the lanes left over after one lane per column go to splitting the
  // next heaviest columns too (by their larger sign, then their size, while
  // that sign exceeds kSignCap - 4), which shrinks the largest lanes that set
  // the warps' step counts
  std::vector<int> pos(cw), neg(cw), rank(cw);
  for (int c = 0; c < cw; ++c) {
    neg[c] = 0;
    for (uint32_t e : cols[c]) neg[c] += (e >> 31) ? 1 : 0;
    pos[c] = (int)cols[c].size() - neg[c];
    if ((int)cols[c].size() > 2 * kLaneCap || pos[c] > 2 * kSignCap || neg[c] > 2 * kSignCap)
      return false;
  }
  std::iota(rank.begin(), rank.end(), 0);
  auto heavy = [&](int c) { return std::max(pos[c], neg[c]) * 4096 + pos[c] + neg[c]; };
  std::stable_sort(rank.begin(), rank.end(), [&](int x, int y) { return heavy(x) > heavy(y); });
  std::vector<char> split(cw, 0);
  int spare = kLanes - cw;
  for (int c = 0; c < cw; ++c)
    if ((int)cols[c].size() > kLaneCap || pos[c] > kSignCap || neg[c] > kSignCap) {
      split[c] = 1;
      --spare;
    }
  if (spare < 0) return false;
  for (int i = 0; i < cw && spare > 0; ++i)
    if (!split[rank[i]] && std::max(pos[rank[i]], neg[rank[i]]) > kSignCap - 4) {
      split[rank[i]] = 1;
      --spare;
    }
  for (int c = 0; c < cw; ++c) {
    const int cnt = (int)cols[c].size();
    const int nparts = split[c] ? 2 : 1;
    // a split column alternates its + entries and its - entries between the parts
    int seen[2] = {0, 0};
    Part pp[2];
    for (int h = 0; h < nparts; ++h) {
      pp[h].col = c;
      pp[h].which = h;
    }
    for (int i = 0; i < cnt; ++i) {
      const uint32_t e = cols[c][i];
      const uint32_t j = e & 0x7FFFFFFFu;
      if (j + kPad > 0xFFFFu) return false;
      const int sg = (e >> 31) ? 1 : 0;
      Part& p = pp[nparts == 2 ? (seen[sg]++ & 1) : 0];
      p.ent[sg].push_back((uint16_t)(j + kPad));
      p.bank[sg][j & 31u] += 1;
    }
    for (int h = 0; h < nparts; ++h) {
      if (pp[h].ent[1].size() > pp[h].ent[0].size()) flip(pp[h]);  // the larger sign in the + phase
      parts.push_back(pp[h]);
    }
  }
  const int V = (int)parts.size();
  if (V > kLanes) return false;
  const int NW = (V + 31) / 32;
  // 2. grouping: a warp takes its steps from its largest lane per sign, so
  // its 32 parts should have about the same number of + entries and of -
  // entries: parts sorted by + count into stripes of kStripe warps, each
  // stripe sorted by - count and cut into warps
  const int stripe = 32 * kStripe;
  std::vector<int> order(V);
  std::iota(order.begin(), order.end(), 0);
  auto cnt = [&](int x, int sg) { return (int)parts[x].ent[sg].size(); };
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cnt(x, 0) > cnt(y, 0); });
  for (int s0 = 0; s0 < V; s0 += stripe)
    std::stable_sort(order.begin() + s0, order.begin() + std::min(V, s0 + stripe),
                     [&](int x, int y) { return cnt(x, 1) > cnt(y, 1); });
  std::vector<WarpSet> ws(kWarps);
  for (auto& w : ws) {
    std::fill(w.lane, w.lane + 32, -1);
    std::fill(&w.bank[0][0], &w.bank[0][0] + 64, 0);
  }
  for (int i = 0; i < V; ++i) {
    WarpSet& w = ws[i / 32];
    w.lane[i % 32] = order[i];
    add_part(parts, w, i % 32, order[i], 1);
  }
  std::vector<int> cost(kWarps, 0);
  for (int w = 0; w < NW; ++w) cost[w] = warp_cost(parts, ws[w]);
  // local search: swap two parts of (nearly) the same +/- counts between two
  // warps, which keeps the warps' largest lanes and reshapes their per-bank
  // loads; a swap is kept when the pair's total step count does not grow
  // (ties half the time), and one warp in two is the currently costliest
  std::vector<int> where(V);  // part -> warp * 32 + lane
  for (int w = 0; w < NW; ++w)
    for (int k = 0; k < 32; ++k)
      if (ws[w].lane[k] >= 0) where[ws[w].lane[k]] = w * 32 + k;
  int pmax = 0;
  for (int i = 0; i < V; ++i) pmax = std::max(pmax, std::max(cnt(i, 0), cnt(i, 1)));
  const int mmax = pmax;
  std::vector<std::vector<int>> shape((pmax + 1) * (mmax + 1));  // parts by (+ count, - count)
  for (int i = 0; i < V; ++i) shape[cnt(i, 0) * (mmax + 1) + cnt(i, 1)].push_back(i);
  Rng rng{0x9E3779B97F4A7C15ull};
  for (int64_t it = 0; NW > 1 && it < search; ++it) {
    int x;
    if (rng.next() & 1u) {
      const int a = (int)(std::max_element(cost.begin(), cost.begin() + NW) - cost.begin());
      x = ws[a].lane[rng.next() & 31u];
      if (x < 0) continue;
    } else {
      x = (int)(rng.next() % (uint32_t)V);
    }
    if ((rng.next() & 7u) == 0) {
      // turn part x around (gather its column negated, or no longer negated)
      const int a = where[x] / 32, i = where[x] % 32;
      WarpSet na = ws[a];
      add_part(parts, na, i, x, -1);
      flip(parts[x]);
      add_part(parts, na, i, x, 1);
      const int ca = warp_cost(parts, na);
      if (ca < cost[a] || (ca == cost[a] && (rng.next() & 1u))) {
        ws[a] = na;
        cost[a] = ca;
        // the part's shape changed: move it to its new shape list
        auto& from = shape[cnt(x, 1) * (mmax + 1) + cnt(x, 0)];
        from.erase(std::find(from.begin(), from.end(), x));
        shape[cnt(x, 0) * (mmax + 1) + cnt(x, 1)].push_back(x);
      } else {
        flip(parts[x]);
      }
      continue;
    }
    const int r = (int)(rng.next() % 9u);
    const int pp = cnt(x, 0) + (r % 3) - 1, mm = cnt(x, 1) + (r / 3) - 1;
    if (pp < 0 || mm < 0 || pp > pmax || mm > mmax) continue;
    const std::vector<int>& cand = shape[pp * (mmax + 1) + mm];
    if (cand.empty()) continue;
    const int y = cand[rng.next() % (uint32_t)cand.size()];
    const int a = where[x] / 32, i = where[x] % 32, b = where[y] / 32, j = where[y] % 32;
    if (a == b) continue;
    WarpSet na = ws[a], nb = ws[b];
    add_part(parts, na, i, x, -1);
    add_part(parts, na, i, y, 1);
    na.lane[i] = y;
    add_part(parts, nb, j, y, -1);
    add_part(parts, nb, j, x, 1);
    nb.lane[j] = x;
    const int ca = warp_cost(parts, na), cb = warp_cost(parts, nb);
    const int d = ca + cb - cost[a] - cost[b];
    if (d < 0 || (d == 0 && (rng.next() & 1u))) {
      ws[a] = na;
      ws[b] = nb;
      cost[a] = ca;
      cost[b] = cb;
      where[x] = b * 32 + j;
      where[y] = a * 32 + i;
    }
  }
  // 3 + 4. colour each phase of each warp and emit the per-lane offsets: the +
  // phase fills register steps [kTT - T+, kTT), the - phase steps [0, T-)
  // (step t of the - phase at register step T- - 1 - t)
  out.words.assign((size_t)kWarps * (kTT / 2) * 32, 0u);
  out.wsteps.assign(kWarps * 2, 0);
  out.slot.assign(kLanes, -1);
  out.steps = 0;
  int nsplit = 0;
  for (int w = 0; w < NW; ++w) {
    const WarpSet& W = ws[w];
    int T[2];
    for (int sg = 0; sg < 2; ++sg) T[sg] = phase_steps(parts, W, sg);
    if (T[0] + T[1] > kTT) return false;
    out.wsteps[2 * w] = T[0];
    out.wsteps[2 * w + 1] = T[1];
    out.steps += T[0] + T[1];
    for (int sg = 0; sg < 2; ++sg) {
      std::vector<int> eu, ev, val, col;
      for (int k = 0; k < 32; ++k) {
        const int pi = W.lane[k];
        if (pi < 0) continue;
        for (uint16_t o : parts[pi].ent[sg]) {
          eu.push_back(k);
          ev.push_back(o & 31);  // row offset kPad + j: bank j mod 32
          val.push_back(o);
        }
      }
      if (T[sg] == 0) continue;
      colour(eu, ev, T[sg], col);
      std::vector<int> at(32 * T[sg], -1);    // at[k T + t]: offset lane k reads at step t
      std::vector<char> used(32 * T[sg], 0);  // used[b T + t]: bank b taken at step t
      for (size_t e = 0; e < eu.size(); ++e) {
        at[eu[e] * T[sg] + col[e]] = val[e];
        used[ev[e] * T[sg] + col[e]] = 1;
      }
      for (int t = 0; t < T[sg]; ++t) {
        int freeb = 0;
        while (freeb < 32 && used[freeb * T[sg] + t]) ++freeb;
        for (int k = 0; k < 32; ++k) {
          int o = at[k * T[sg] + t];
          if (o < 0) o = freeb < 32 ? freeb : 0;  // the zero pad element of a free bank
          const int r = sg == 0 ? kTT - T[0] + t : T[1] - 1 - t;
          uint32_t& word = out.words[((size_t)w * (kTT / 2) + (r >> 1)) * 32 + k];
          word |= (uint32_t)o << ((r & 1) ? 17 : 0);
        }
      }
    }
    for (int k = 0; k < 32; ++k) {
      const int pi = W.lane[k];
      if (pi < 0) continue;
      const int negf = parts[pi].neg ? (kLanes << 16) : 0;
      if (parts[pi].which == 0) {
        out.slot[w * 32 + k] = parts[pi].col | negf;
      } else {
        out.slot[w * 32 + k] = (cw + nsplit) | negf;
        out.partner[parts[pi].col] = cw + nsplit;
        ++nsplit;
      }
    }
  }
  return cw + nsplit <= kLanes;
}

}  // namespace sched
}  // namespace spm
