// Pair schedule of the exchange (host only, no CUDA): batches of pairs (i, j) whose pair fields
// share one scratch slot each, and per batch the targets with the contributions (pair slot,
// partner orbital, occupation index, conjugation) each target accumulates.
//
// (V_x tgt_j) = -sum_i d_i src_i v_ij with v_ij = IFFT[K FFT[conj(src_i) tgt_j]] (Eq. vxdiag).
// Orbitals are taken in tiles of B.  Symmetric case (tgt = src): tiles I <= J and pairs i <= j
// inside diagonal tiles; the pair (i, j) feeds target j with partner i and, when i != j, target
// i with partner j through v_ji = conj(v_ij) (the kernel is real and even).  General case: every
// (i, j) pair of an I x J tile feeds target j.  A target's first batch overwrites it, later
// batches accumulate.
#pragma once

#include <algorithm>
#include <map>
#include <vector>

namespace pt {

struct PairDesc {
  int i, j;    // source index, target index
  int o1, o2;  // occupation indices of its contributions (o2 < 0: a single one)
};
struct TargetDesc {
  int t, cbeg, cend, first;
};
struct Contrib {
  int slot, partner, occ, conj;
};

struct PairPlan {
  int N = 0, M = 0, B = 0;
  bool sym = false;
  std::vector<int> pair_off, tgt_off;  // per batch offsets (size nbatch + 1)
  std::vector<PairDesc> pairs;
  std::vector<TargetDesc> tgts;
  std::vector<Contrib> contribs;
  int max_pairs = 0, max_tgts = 0;
};

inline PairPlan plan_pairs(int N, int M, bool sym, int B) {
  PairPlan s;
  s.N = N;
  s.M = M;
  s.B = B;
  s.sym = sym;
  std::vector<char> touched(sym ? N : M, 0);
  s.pair_off.push_back(0);
  s.tgt_off.push_back(0);
  auto finish_batch = [&](std::map<int, std::vector<Contrib>>& per_t) {
    for (auto& kv : per_t) {
      TargetDesc td;
      td.t = kv.first;
      td.cbeg = int(s.contribs.size());
      for (auto& c : kv.second) s.contribs.push_back(c);
      td.cend = int(s.contribs.size());
      td.first = touched[kv.first] ? 0 : 1;
      touched[kv.first] = 1;
      s.tgts.push_back(td);
    }
    s.max_pairs = std::max(s.max_pairs, int(s.pairs.size()) - s.pair_off.back());
    s.max_tgts = std::max(s.max_tgts, int(s.tgts.size()) - s.tgt_off.back());
    s.pair_off.push_back(int(s.pairs.size()));
    s.tgt_off.push_back(int(s.tgts.size()));
  };
  if (sym) {
    const int nb = (N + B - 1) / B;
    for (int J = 0; J < nb; ++J) {
      for (int I = 0; I <= J; ++I) {
        std::map<int, std::vector<Contrib>> per_t;
        const int base = int(s.pairs.size());
        const int i0 = I * B, i1 = std::min(N, i0 + B), j0 = J * B, j1 = std::min(N, j0 + B);
        for (int i = i0; i < i1; ++i) {
          for (int j = (I == J ? i : j0); j < j1; ++j) {
            const int slot = int(s.pairs.size()) - base;
            s.pairs.push_back({i, j, i, i == j ? -1 : j});
            per_t[j].push_back({slot, i, i, 0});
            if (i != j) per_t[i].push_back({slot, j, j, 1});
          }
        }
        finish_batch(per_t);
      }
    }
  } else {
    const int nbi = (N + B - 1) / B, nbj = (M + B - 1) / B;
    for (int J = 0; J < nbj; ++J) {
      for (int I = 0; I < nbi; ++I) {
        std::map<int, std::vector<Contrib>> per_t;
        const int base = int(s.pairs.size());
        const int i0 = I * B, i1 = std::min(N, i0 + B), j0 = J * B, j1 = std::min(M, j0 + B);
        for (int j = j0; j < j1; ++j) {
          for (int i = i0; i < i1; ++i) {
            const int slot = int(s.pairs.size()) - base;
            s.pairs.push_back({i, j, i, -1});
            per_t[j].push_back({slot, i, i, 0});
          }
        }
        finish_batch(per_t);
      }
    }
  }
  return s;
}

}  // namespace pt
