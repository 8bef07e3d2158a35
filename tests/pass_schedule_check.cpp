// Host check of the fused-pass schedule (built by the test from the library's
// planner source; no GPU).  For a generated grid circuit, every qubit's events in
// the schedule of its half (all levels, all passes, in order) must be the circuit's
// events on that qubit: the same non-diagonal gates in the same order, and between
// two of them the same multiset of diagonal terms (T, CZ with its partner, cut slot
// with its copy bit and type).  Diagonal terms commute with each other, so only
// their multiset between gates is fixed.
//
// usage: pass_schedule_check R C depth seed cut_row fuse pass_order
// prints "ok <passes upper> <passes lower>" or the first difference; exit 0 / 1.
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

int main(int argc, char** argv) {
  if (argc != 8) {
    fprintf(stderr, "usage: R C depth seed cut_row fuse pass_order\n");
    return 2;
  }
  const int R = atoi(argv[1]), C = atoi(argv[2]), depth = atoi(argv[3]);
  const uint64_t seed = strtoull(argv[4], nullptr, 10);
  const int b = atoi(argv[5]), fuse = atoi(argv[6]), order = atoi(argv[7]);
  Circuit circ;
  std::string err = generate_circuit(R, C, depth, seed, b, circ, 0);
  if (!err.empty()) {
    printf("generate: %s\n", err.c_str());
    return 1;
  }
  CutPlan plan;
  err = build_cut_plan(circ, b, fuse, plan, order);
  if (!err.empty()) {
    printf("plan: %s\n", err.c_str());
    return 1;
  }
  const int nu = plan.n_u;
  std::map<std::pair<int, int>, int> bit_of;  // (layer, upper qubit) -> copy bit
  for (int m = 0; m < plan.c; ++m) bit_of[{plan.cuts[m].t, plan.cuts[m].h}] = m;
  int npass[2] = {0, 0};
  for (int h = 0; h < 2; ++h) {
    const int n = h ? plan.n_l : plan.n_u;
    const int off = h ? nu : 0;
    // the circuit's events per qubit of this half, layer by layer
    std::vector<std::vector<Ev>> want(n);
    bool uniform = true;  // layer 0: H on every qubit (generated circuits)
    for (const Gate& g : circ.gates) {
      const bool in1 = g.q1 >= off && g.q1 < off + n;
      const bool in2 = g.q2 >= off && g.q2 < off + n;
      if (g.code == G_CZ) {
        if (in1 && in2) {
          want[g.q1 - off].push_back({false, "CZ" + std::to_string(g.q2 - off)});
          want[g.q2 - off].push_back({false, "CZ" + std::to_string(g.q1 - off)});
        } else if (in1 || in2) {
          const int m = bit_of.at({g.t, std::min(g.q1, g.q2)});
          const bool lower_end = (h == 1);
          const int q = in1 ? g.q1 - off : g.q2 - off;
          want[q].push_back({false, std::string(lower_end ? "Z" : "P") + std::to_string(m)});
        }
      } else if (in1) {
        if (g.code == G_T)
          want[g.q1 - off].push_back({false, "T"});
        else if (!(g.t == 0 && uniform && g.code == G_H))
          want[g.q1 - off].push_back({true, std::to_string(g.code)});
      }
    }
    // the schedule's events per qubit
    std::vector<std::vector<Ev>> got(n);
    const HalfSchedule& S = plan.sched[h];
    for (const Level& L : S.levels)
      for (const PassDesc& p : L.passes) {
        ++npass[h];
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
    for (int q = 0; q < n; ++q) {
      const auto a = canonical(want[q]), bb = canonical(got[q]);
      if (a != bb) {
        printf("half %d qubit %d differs: want", h, q);
        for (auto& x : a) printf(" %s", x.c_str());
        printf(" | got");
        for (auto& x : bb) printf(" %s", x.c_str());
        printf("\n");
        return 1;
      }
    }
  }
  printf("ok %d %d\n", npass[0], npass[1]);
  return 0;
}
