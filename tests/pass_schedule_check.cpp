// Host check of the fused-pass schedule (built by the test from the library's
// planner source; no GPU).  For a generated grid circuit, every qubit's events in
// the schedule of its half (all levels, all passes, in order) must be the circuit's
// events on that qubit: the same non-diagonal gates in the same order, and between
// two of them the same multiset of diagonal terms (T, CZ with its partner, cut slot
// with its copy bit and type).  Diagonal terms commute with each other, so only
// their multiset between gates is fixed.
//
// usage: pass_schedule_check R C depth seed cut_row fuse pass_order [phase]
//        pass_schedule_check R C depth seed multi fuse pass_order r1 [r2 ...]
// With "phase" the plan turns the cut CZs that commute to the end of the circuit
// (no non-diagonal gate on either qubit afterwards) into output signs; they then
// leave the halves' events.
// The second form checks every part of a multi-part cut at rows r1 < r2 < ...
// (P_l slots for the boundary below a part, Z^l for the one above, with the part's
// own copy bits).  Prints "ok <passes per half or part>" or the first difference;
// exit 0 / 1.
#include "../paper_1802_06952_gb300/csrc/host.cpp"

#include <cstdio>
#include <cstdlib>
#include <string>
#include <vector>

using namespace sim;

namespace {

// one event on a qubit: a gate (code), or a diagonal term
struct Ev {
  bool gate;
  std::string what;
};

// per-qubit sequences -> list of segments: each gate, and between gates the sorted
// diagonal terms
std::vector<std::string> canonical(const std::vector<Ev>& evs) {
  std::vector<std::string> out, diag;
  auto flush = [&]() {
    std::sort(diag.begin(), diag.end());
    std::string s = "D{";
    for (auto& d : diag) s += d + ",";
    out.push_back(s + "}");
    diag.clear();
  };
  for (const Ev& e : evs) {
    if (e.gate) {
      flush();
      out.push_back("G" + e.what);
    } else {
      diag.push_back(e.what);
    }
  }
  flush();
  return out;
}

}  // namespace

// schedule events per qubit of one half-circuit or part
std::vector<std::vector<Ev>> schedule_events(const HalfSchedule& S, int n, int& npass) {
  std::vector<std::vector<Ev>> got(n);
  for (const Level& L : S.levels)
    for (const PassDesc& p : L.passes) {
      ++npass;
      for (int o = p.op_begin; o < p.op_begin + p.op_count; ++o) {
        const OpRec& op = S.ops[o];
        if (op.type == OP_GATE) {
          const int code = op.kind == 1 ? G_X2 : op.kind == 2 ? G_Y2 : op.kind == 3 ? G_H : -1;
          got[op.q].push_back({true, std::to_string(code)});
        } else if (op.type == OP_DIAG) {
          for (int q = 0; q < n; ++q)
            if ((op.tmask >> q) & 1u) got[q].push_back({false, "T"});
          for (int s = 0; s < op.nsh; ++s)
            for (int a = 0; a < n; ++a)
              if ((op.sh_m[s] >> a) & 1u) {
                const int c2 = a + (int)op.sh_d[s];
                got[a].push_back({false, "CZ" + std::to_string(c2)});
                got[c2].push_back({false, "CZ" + std::to_string(a)});
              }
          for (int i = 0; i < op.ncut; ++i) {
            const bool z = (op.cutz >> i) & 1u;
            got[op.cutq[i]].push_back({false, std::string(z ? "Z" : "P") + std::to_string(op.cutm[i])});
          }
        }
      }
    }
  return got;
}

bool same(const std::vector<std::vector<Ev>>& want, const std::vector<std::vector<Ev>>& got, int part) {
  for (size_t q = 0; q < want.size(); ++q) {
    const auto a = canonical(want[q]), bb = canonical(got[q]);
    if (a != bb) {
      printf("part %d qubit %zu differs: want", part, q);
      for (auto& x : a) printf(" %s", x.c_str());
      printf(" | got");
      for (auto& x : bb) printf(" %s", x.c_str());
      printf("\n");
      return false;
    }
  }
  return true;
}

int check_multi(const Circuit& circ, const std::vector<int>& rows, int fuse, int order) {
  MultiPlan mp;
  std::string err = build_multi_plan(circ, rows, fuse, order, mp);
  if (!err.empty()) {
    printf("plan: %s\n", err.c_str());
    return 1;
  }
  std::vector<int> part_of(circ.n);
  for (int p = 0; p < mp.t; ++p)
    for (int q = mp.offset[p]; q < mp.offset[p] + mp.nq[p]; ++q) part_of[q] = p;
  // cut CZs per boundary in (layer, upper qubit) order -> (boundary, bit)
  std::vector<std::vector<std::pair<int, int>>> cuts(mp.t);
  for (const Gate& g : circ.gates)
    if (g.code == G_CZ && part_of[g.q1] != part_of[g.q2]) cuts[part_of[g.q2]].push_back({g.t, g.q1});
  std::map<std::pair<int, int>, std::pair<int, int>> where;
  for (int j = 1; j < mp.t; ++j) {
    std::sort(cuts[j].begin(), cuts[j].end());
    for (size_t i = 0; i < cuts[j].size(); ++i) where[cuts[j][i]] = {j, (int)i};
  }
  std::string counts;
  for (int p = 0; p < mp.t; ++p) {
    std::map<std::pair<int, int>, int> local;
    for (size_t m = 0; m < mp.slot_bits[p].size(); ++m) local[mp.slot_bits[p][m]] = (int)m;
    const int n = mp.nq[p], off = mp.offset[p];
    std::vector<std::vector<Ev>> want(n);
    for (const Gate& g : circ.gates) {
      const bool in1 = part_of[g.q1] == p;
      const bool in2 = g.q2 >= 0 && part_of[g.q2] == p;
      if (g.code == G_CZ) {
        if (in1 && in2) {
          want[g.q1 - off].push_back({false, "CZ" + std::to_string(g.q2 - off)});
          want[g.q2 - off].push_back({false, "CZ" + std::to_string(g.q1 - off)});
        } else if (in1 || in2) {
          const int m = local.at(where.at({g.t, g.q1}));
          if (in1)
            want[g.q1 - off].push_back({false, "P" + std::to_string(m)});  // upper end
          else
            want[g.q2 - off].push_back({false, "Z" + std::to_string(m)});  // lower end
        }
      } else if (in1) {
        if (g.code == G_T)
          want[g.q1 - off].push_back({false, "T"});
        else if (!(g.t == 0 && g.code == G_H))
          want[g.q1 - off].push_back({true, std::to_string(g.code)});
      }
    }
    int np = 0;
    if (!same(want, schedule_events(mp.part[p].sched[0], n, np), p)) return 1;
    counts += " " + std::to_string(np);
  }
  printf("ok%s\n", counts.c_str());
  return 0;
}

int main(int argc, char** argv) {
  if (argc < 8) {
    fprintf(stderr, "usage: R C depth seed cut_row|multi fuse pass_order [rows]\n");
    return 2;
  }
  const int R = atoi(argv[1]), C = atoi(argv[2]), depth = atoi(argv[3]);
  const uint64_t seed = strtoull(argv[4], nullptr, 10);
  if (std::string(argv[5]) == "multi") {
    std::vector<int> rows;
    for (int i = 8; i < argc; ++i) rows.push_back(atoi(argv[i]));
    if (rows.empty()) return 2;
    Circuit circ;
    std::string err = generate_circuit(R, C, depth, seed, rows[0], circ, 0);
    if (!err.empty()) {
      printf("generate: %s\n", err.c_str());
      return 1;
    }
    return check_multi(circ, rows, atoi(argv[6]), atoi(argv[7]));
  }
  if (argc != 8 && !(argc == 9 && std::string(argv[8]) == "phase")) return 2;
  const bool phase = argc == 9;
  const int b = atoi(argv[5]), fuse = atoi(argv[6]), order = atoi(argv[7]);
  Circuit circ;
  std::string err = generate_circuit(R, C, depth, seed, b, circ, 0);
  if (!err.empty()) {
    printf("generate: %s\n", err.c_str());
    return 1;
  }
  CutPlan plan;
  err = build_cut_plan(circ, b, fuse, plan, order, phase);
  if (!err.empty()) {
    printf("plan: %s\n", err.c_str());
    return 1;
  }
  const int nu = plan.n_u;
  // cut CZs that commute to the end: no non-diagonal gate on either qubit later
  std::vector<int> last(circ.n, -1);
  for (const Gate& g : circ.gates)
    if (g.code != G_T && g.code != G_CZ) last[g.q1] = std::max(last[g.q1], g.t);
  std::set<std::pair<int, int>> signs;  // (layer, upper qubit)
  if (phase)
    for (const Gate& g : circ.gates)
      if (g.code == G_CZ && g.q1 < nu && g.q2 >= nu && last[g.q1] < g.t && last[g.q2] < g.t && signs.size() < 32)
        signs.insert({g.t, g.q1});
  if ((int)signs.size() != (int)plan.out_cz.size()) {
    printf("output signs: want %zu, plan has %zu\n", signs.size(), plan.out_cz.size());
    return 1;
  }
  std::map<std::pair<int, int>, int> bit_of;  // (layer, upper qubit) -> copy bit
  for (int m = 0; m < plan.c; ++m) bit_of[{plan.cuts[m].t, plan.cuts[m].h}] = m;
  int npass[2] = {0, 0};
  for (int h = 0; h < 2; ++h) {
    const int n = h ? plan.n_l : plan.n_u;
    const int off = h ? nu : 0;
    // the circuit's events per qubit of this half, layer by layer
    std::vector<std::vector<Ev>> want(n);
    for (const Gate& g : circ.gates) {
      const bool in1 = g.q1 >= off && g.q1 < off + n;
      const bool in2 = g.q2 >= off && g.q2 < off + n;
      if (g.code == G_CZ) {
        if (in1 && in2) {
          want[g.q1 - off].push_back({false, "CZ" + std::to_string(g.q2 - off)});
          want[g.q2 - off].push_back({false, "CZ" + std::to_string(g.q1 - off)});
        } else if ((in1 || in2) && !signs.count({g.t, std::min(g.q1, g.q2)})) {
          const int m = bit_of.at({g.t, std::min(g.q1, g.q2)});
          const bool lower_end = (h == 1);
          const int q = in1 ? g.q1 - off : g.q2 - off;
          want[q].push_back({false, std::string(lower_end ? "Z" : "P") + std::to_string(m)});
        }
      } else if (in1) {
        if (g.code == G_T)
          want[g.q1 - off].push_back({false, "T"});
        else if (!(g.t == 0 && g.code == G_H))  // layer 0 (H everywhere) is the initial state
          want[g.q1 - off].push_back({true, std::to_string(g.code)});
      }
    }
    if (!same(want, schedule_events(plan.sched[h], n, npass[h]), h)) return 1;
  }
  printf("ok %d %d\n", npass[0], npass[1]);
  return 0;
}
