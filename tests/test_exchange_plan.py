"""The exchange's pair schedule (csrc/exchange_plan.h, host-only C++) is compiled with the host C++
compiler and checked on the CPU: every pair of the sum appears exactly once, each target receives
every source's contribution exactly once (with the conjugate pair field where the symmetric
schedule reuses v_ji = conj(v_ij)), batches stay inside one B x B tile, slots index their own
batch, and a target's first batch overwrites it while later batches accumulate."""
import collections
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2501_03061_gb300", "csrc")

DRIVER = r"""
#include <cstdio>
#include <cstdlib>
#include "exchange_plan.h"
int main(int argc, char** argv) {
  const int N = std::atoi(argv[1]), M = std::atoi(argv[2]), sym = std::atoi(argv[3]), B = std::atoi(argv[4]);
  const pt::PairPlan p = pt::plan_pairs(N, M, sym != 0, B);
  std::printf("m %d %d\n", p.max_pairs, p.max_tgts);
  for (size_t b = 0; b < p.pair_off.size(); ++b) std::printf("o %d %d\n", p.pair_off[b], p.tgt_off[b]);
  for (const auto& q : p.pairs) std::printf("p %d %d %d %d\n", q.i, q.j, q.o1, q.o2);
  for (const auto& t : p.tgts) std::printf("t %d %d %d %d\n", t.t, t.cbeg, t.cend, t.first);
  for (const auto& c : p.contribs) std::printf("c %d %d %d %d\n", c.slot, c.partner, c.occ, c.conj);
  return 0;
}
"""


@pytest.fixture(scope="module")
def planner(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("plan")
    src = d / "plan.cpp"
    src.write_text(DRIVER)
    exe = d / "plan"
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", CSRC, str(src), "-o", str(exe)], check=True)

    def run(N, M, sym, B):
        out = subprocess.run([str(exe), str(N), str(M), str(int(sym)), str(B)], capture_output=True, text=True,
                             check=True).stdout.split("\n")
        rec = collections.defaultdict(list)
        for line in out:
            if line:
                k, *v = line.split()
                rec[k].append(tuple(int(x) for x in v))
        return rec
    return run


@pytest.mark.parametrize("N,M,sym,B", [
    (1, 1, True, 1), (7, 7, True, 2), (13, 13, True, 6), (23, 23, True, 10), (320, 320, True, 16),
    (33, 33, True, 16), (5, 5, True, 16), (7, 5, False, 2), (12, 8, False, 6), (9, 20, False, 4),
    (1, 3, False, 16),
])
def test_schedule_covers_the_exchange_sum_once(planner, N, M, sym, B):
    r = planner(N, M, sym, B)
    (max_pairs, max_tgts), = r["m"]
    offs = r["o"]
    pairs, tgts, cons = r["p"], r["t"], r["c"]
    T = N if sym else M
    # every pair exactly once
    want = {(i, j) for i in range(N) for j in range(i if sym else 0, T)} if sym else \
        {(i, j) for i in range(N) for j in range(M)}
    got = [(i, j) for i, j, _, _ in pairs]
    assert len(got) == len(set(got)) and set(got) == want
    for i, j, o1, o2 in pairs:
        assert o1 == i and o2 == (j if sym and i != j else -1)
    # batch offsets
    assert offs[0] == (0, 0) and offs[-1] == (len(pairs), len(tgts))
    assert all(a[0] <= b[0] and a[1] <= b[1] for a, b in zip(offs, offs[1:]))
    sizes = [b[0] - a[0] for a, b in zip(offs, offs[1:])]
    assert max_pairs == max(sizes) and max_pairs <= B * B
    assert max_tgts == max(b[1] - a[1] for a, b in zip(offs, offs[1:]))
    # capacities of the 64^3 path's parameter block for tiles up to 16: B^2 pairs, 2B targets and
    # 2 B^2 contributions per batch
    assert max_tgts <= 2 * B
    for a, b in zip(offs, offs[1:]):
        if b[1] > a[1]:
            assert tgts[b[1] - 1][2] - tgts[a[1]][1] <= 2 * B * B
    seen = set()
    total = collections.Counter()
    for (p0, t0), (p1, t1) in zip(offs, offs[1:]):
        bp = pairs[p0:p1]
        # one B x B tile per batch
        assert len({i // B for i, _, _, _ in bp}) == 1 and len({j // B for _, j, _, _ in bp}) == 1
        expect = collections.defaultdict(list)
        for slot, (i, j, _, _) in enumerate(bp):
            expect[j].append((slot, i, i, 0))
            if sym and i != j:
                expect[i].append((slot, j, j, 1))
        bt = tgts[t0:t1]
        assert [t for t, _, _, _ in bt] == sorted(expect)  # each target of the batch once, in order
        for t, cb, ce, first in bt:
            assert sorted(cons[cb:ce]) == sorted(expect[t])
            assert first == (t not in seen)
            seen.add(t)
            for slot, partner, occ, conj in cons[cb:ce]:
                assert 0 <= slot < p1 - p0
                total[(t, partner, conj)] += 1
    # the full sum: each target receives each source once; with symmetric pairs the source k
    # reaches target t through v_kt (k <= t) or through conj(v_tk) (k > t)
    assert seen == set(range(T))
    if sym:
        assert total == collections.Counter({(t, k, int(k > t)): 1 for t in range(N) for k in range(N)})
    else:
        assert total == collections.Counter({(t, k, 0): 1 for t in range(M) for k in range(N)})
    # contribution ranges tile the contribution table
    assert [(cb, ce) for _, cb, ce, _ in tgts] == list(zip([0] + [ce for _, _, ce, _ in tgts[:-1]],
                                                           [ce for _, _, ce, _ in tgts]))
