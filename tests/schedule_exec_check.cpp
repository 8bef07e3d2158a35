// Host execution of the fused-pass schedule (built by the test from the library's
// planner source; no GPU).  For a circuit given as a gate list, every half of each
// listed copy is evolved through its schedule in FP64: the levels of the copy tree
// in order, their passes in order, each op with its full 2x2 matrix (GATE) or its
// combined diagonal (DIAG: T, CZ and cut-slot terms at the copy's bits), the first
// pass starting from |0...0> or from the uniform state of the omitted H layer.
// The test compares the resulting leaves with the oracle's half-states.
//
// It also evaluates the sparse leaf entries as the library defines them: for every
// number d of trailing levels whose ops act non-diagonally on at most 10 qubits Q,
// the selected entries of a leaf from its ancestor d levels up, by applying those
// levels' ops to the 2^|Q| ancestor entries that agree with the entry outside Q,
// and reports the largest difference from the leaf's own entries.
//
// usage: schedule_exec_check gate_list_file cut_row fuse pass_order out_file k1 [k2 ...]
//        schedule_exec_check gate_list_file multi:r1,r2,... fuse pass_order out_file k1 [k2 ...]
// Writes, per listed copy, the upper then the lower leaf (complex128, index order)
// to out_file and prints "ok <sparse depths tried> <max sparse difference>".  The
// multi form evolves every part of a multi-part cut at rows r1 < r2 < ... (each
// part's schedule with its own copy index k, skipped where k >= 2^{c_p}) and writes
// the parts' states in order.
#include "../paper_1802_06952_gb300/csrc/host.cpp"

#include <complex>
#include <cstdio>
#include <cstring>
#include <cstdlib>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

using namespace sim;
using cd = std::complex<double>;

namespace {

cd omega(int e) {
  const double r = 0.70710678118654752440;
  static const cd w[8] = {cd(1, 0), cd(r, r), cd(0, 1), cd(-r, r), cd(-1, 0), cd(-r, -r), cd(0, -1), cd(r, -r)};
  return w[e & 7];
}

// exponent of w (mod 8) of a DIAG op at index x for copy k, and its projector test
int diag_exponent(const OpRec& op, uint64_t x, uint64_t k, bool& keep) {
  int e = __builtin_popcountll(x & op.tmask);
  int s2 = 0;
  for (int s = 0; s < op.nsh; ++s) s2 += __builtin_popcountll(x & (x >> op.sh_d[s]) & op.sh_m[s]);
  e += 4 * s2;
  keep = true;
  for (int i = 0; i < op.ncut; ++i) {
    const uint64_t bit = (x >> op.cutq[i]) & 1ull;
    const uint64_t l = (k >> op.cutm[i]) & 1ull;
    if (!((op.cutz >> i) & 1u)) {
      if (bit != l) keep = false;  // P_l on this qubit
    } else if (l && bit) {
      e += op.cutw[i];  // phase slot w^{weight l x}
    }
  }
  return e & 7;
}

void apply_gate(const OpRec& op, std::vector<cd>& psi, int local_bit) {
  const cd m00(op.md[0], op.md[1]), m01(op.md[2], op.md[3]), m10(op.md[4], op.md[5]), m11(op.md[6], op.md[7]);
  const uint64_t b = 1ull << local_bit;
  for (uint64_t i = 0; i < psi.size(); ++i)
    if (!(i & b)) {
      const cd a0 = psi[i], a1 = psi[i | b];
      psi[i] = m00 * a0 + m01 * a1;
      psi[i | b] = m10 * a0 + m11 * a1;
    }
}

// the ops of levels [j0, j1) in order
std::vector<const OpRec*> ops_of(const HalfSchedule& S, int j0, int j1) {
  std::vector<const OpRec*> out;
  for (int j = j0; j < j1; ++j)
    for (const PassDesc& pd : S.levels[j].passes)
      for (int o = pd.op_begin; o < pd.op_begin + pd.op_count; ++o) out.push_back(&S.ops[o]);
  return out;
}

// the state of copy k after levels [0, upto)
std::vector<cd> evolve(const HalfSchedule& S, uint64_t k, int upto) {
  const int n = S.n;
  std::vector<cd> psi((size_t)1 << n, cd(0, 0));
  const PassDesc& first = S.levels[0].passes[0];
  if (first.src == SRC_UNIFORM)
    for (auto& a : psi) a = cd(std::pow(2.0, -0.5 * n), 0);
  else
    psi[0] = cd(1, 0);
  for (const OpRec* op : ops_of(S, 0, upto)) {
    if (op->type == OP_SWAP) continue;
    if (op->type == OP_GATE) {
      if (op->cond >= 0 && !((k >> op->cond) & 1ull)) continue;
      apply_gate(*op, psi, op->q);
    } else {
      for (uint64_t x = 0; x < psi.size(); ++x) {
        bool keep;
        const int e = diag_exponent(*op, x, k, keep);
        psi[x] = keep ? psi[x] * omega(e) : cd(0, 0);
      }
    }
  }
  return psi;
}

}  // namespace

int main(int argc, char** argv) {
  if (argc < 7) {
    fprintf(stderr, "usage: %s gate_list_file cut_row fuse pass_order out_file k1 [k2 ...]\n", argv[0]);
    return 2;
  }
  std::ifstream in(argv[1]);
  std::stringstream ss;
  ss << in.rdbuf();
  Circuit c;
  std::string err = parse_circuit(ss.str().c_str(), c);
  if (!err.empty()) {
    printf("parse: %s\n", err.c_str());
    return 1;
  }
  FILE* out = fopen(argv[5], "wb");
  if (!out) return 1;
  if (strncmp(argv[2], "multi:", 6) == 0) {
    std::vector<int> rows;
    for (const char* p = argv[2] + 6; *p;) {
      rows.push_back((int)strtol(p, (char**)&p, 10));
      if (*p == ',') ++p;
    }
    MultiPlan mp;
    err = build_multi_plan(c, rows, atoi(argv[3]), atoi(argv[4]), mp);
    if (!err.empty()) {
      printf("plan: %s\n", err.c_str());
      return 1;
    }
    for (int a = 6; a < argc; ++a) {
      const uint64_t k = strtoull(argv[a], nullptr, 10);
      for (int p = 0; p < mp.t; ++p) {
        const HalfSchedule& S = mp.part[p].sched[0];
        if (k >> mp.slot_bits[p].size()) continue;
        const std::vector<cd> st = evolve(S, k, (int)S.levels.size());
        fwrite(st.data(), sizeof(cd), st.size(), out);
      }
    }
    fclose(out);
    printf("ok 0 0\n");
    return 0;
  }
  CutPlan P;
  err = build_cut_plan(c, atoi(argv[2]), atoi(argv[3]), P, atoi(argv[4]), false);
  if (!err.empty()) {
    printf("plan: %s\n", err.c_str());
    return 1;
  }
  int depths_tried = 0;
  double worst = 0;
  for (int a = 6; a < argc; ++a) {
    const uint64_t k = strtoull(argv[a], nullptr, 10);
    for (int h = 0; h < 2; ++h) {
      const HalfSchedule& S = P.sched[h];
      const int J = (int)S.levels.size();
      const std::vector<cd> leaf = evolve(S, k, J);
      fwrite(leaf.data(), sizeof(cd), leaf.size(), out);
      // sparse entries from the ancestor d levels up, on a seeded selection
      for (int d = 1; d < J; ++d) {
        uint32_t qmask = 0;
        for (const OpRec* op : ops_of(S, J - d, J))
          if (op->type == OP_GATE) qmask |= 1u << op->q;
        std::vector<int> qpos;
        for (int q = 0; q < S.n; ++q)
          if ((qmask >> q) & 1u) qpos.push_back(q);
        if (qpos.size() > (size_t)kMaxSparseQ) continue;
        ++depths_tried;
        const std::vector<cd> anc = evolve(S, k, J - d);
        const std::vector<const OpRec*> tail = ops_of(S, J - d, J);
        uint64_t state = 0x9E3779B97F4A7C15ull ^ (k * 2 + h) ^ ((uint64_t)d << 40);
        for (int s = 0; s < 16; ++s) {
          const uint64_t x = splitmix64_next(state) & ((1ull << S.n) - 1);
          const uint64_t xo = x & ~(uint64_t)qmask;
          std::vector<cd> v((size_t)1 << qpos.size());
          std::vector<uint64_t> idx(v.size());
          for (size_t y = 0; y < v.size(); ++y) {
            uint64_t off = 0;
            for (size_t b = 0; b < qpos.size(); ++b)
              if ((y >> b) & 1) off |= 1ull << qpos[b];
            idx[y] = xo | off;
            v[y] = anc[idx[y]];
          }
          for (const OpRec* op : tail) {
            if (op->type == OP_SWAP) continue;
            if (op->type == OP_GATE) {
              if (op->cond >= 0 && !((k >> op->cond) & 1ull)) continue;
              int lb = 0;
              while (qpos[lb] != op->q) ++lb;
              apply_gate(*op, v, lb);
            } else {
              for (size_t y = 0; y < v.size(); ++y) {
                bool keep;
                const int e = diag_exponent(*op, idx[y], k, keep);
                v[y] = keep ? v[y] * omega(e) : cd(0, 0);
              }
            }
          }
          uint64_t ex = 0;
          for (size_t b = 0; b < qpos.size(); ++b)
            if ((x >> qpos[b]) & 1ull) ex |= 1ull << b;
          worst = std::max(worst, std::abs(v[ex] - leaf[x]));
        }
      }
    }
  }
  fclose(out);
  printf("ok %d %.3e\n", depths_tried, worst);
  return 0;
}
