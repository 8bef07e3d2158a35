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
// It also recomputes, for every pass the register-blocked sweep runs, what that
// kernel derives from the host's per-op tables, and compares it with the op in
// qubit space for every index: each gate's rank under the pass's rank map (moved by
// its warp/register exchanges) is the gate's qubit; the gate's unscaled update times
// the common factor is its matrix; a diagonal op's exponent built as the kernel
// builds it (thread part, register-part table, register partners B, cut slots,
// the pass phase) equals the qubit-space exponent mod 8, with the same projector
// test; sign-only ops have exponents 0 or 4; and the pass's scale and phase are the
// product of the factors its unscaled gates leave out.
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

// the register-blocked sweep's view of one pass, checked against qubit space for
// copy k; returns an empty string or the first difference
std::string check_register_pass(const HalfSchedule& S, const PassDesc& p, uint64_t k) {
  const int R = p.k - 8;
  int ord[16];
  for (int r = 0; r < 16; ++r) ord[r] = r < p.k ? p.order[r] : -1;
  const double s2 = 0.70710678118654752440;
  const cd fxy(0.5, 0.5);  // (1+i)/2: X^1/2, Y^1/2 without it are [[1,-i],[-i,1]], [[1,-1],[1,1]]
  int n_xy = 0, n_h = 0;
  char buf[256];
  for (int oi = 0; oi < p.op_count; ++oi) {
    const OpRec& op = S.ops[p.op_begin + oi];
    if (op.type == OP_SWAP) {
      for (int m = 0; m < 3; ++m) std::swap(ord[5 + m], ord[10 + m]);
      for (int r = 0; r < 8; ++r)
        if (op.tq[r] != ord[r]) return "swap: thread rank map";
      continue;
    }
    if (op.type == OP_GATE) {
      if (op.lq < 0 || op.lq >= p.k || ord[op.lq] != op.q) {
        snprintf(buf, sizeof buf, "gate on qubit %d at rank %d holding %d", op.q, op.lq, op.lq >= 0 ? ord[op.lq] : -1);
        return buf;
      }
      cd u[4];
      if (op.kind == 1) {
        u[0] = fxy; u[1] = fxy * cd(0, -1); u[2] = fxy * cd(0, -1); u[3] = fxy;
        ++n_xy;
      } else if (op.kind == 2) {
        u[0] = fxy; u[1] = -fxy; u[2] = fxy; u[3] = fxy;
        ++n_xy;
      } else if (op.kind == 3) {
        u[0] = s2; u[1] = s2; u[2] = s2; u[3] = -s2;
        ++n_h;
      } else {
        return "a general gate in a register-blocked pass";
      }
      for (int e = 0; e < 4; ++e)
        if (std::abs(u[e] - cd(op.md[2 * e], op.md[2 * e + 1])) > 1e-15) return "gate kind and matrix differ";
      continue;
    }
    uint32_t regmask = 0;
    for (int r = 0; r < R; ++r) {
      regmask |= 1u << ord[8 + r];
      if (op.rq[r] != ord[8 + r]) return "diag: register qubits";
    }
    if (op.regmask != regmask) return "diag: register mask";
    const int phase = (oi == p.phase_op) ? p.phase_e : 0;
    if (op.sign_only && phase) return "sign-only op takes the pass phase";
    for (uint64_t x = 0; x < ((uint64_t)1 << S.n); ++x) {
      const uint32_t xt = (uint32_t)x & ~regmask;
      uint32_t j = 0;
      for (int r = 0; r < R; ++r)
        if ((x >> ord[8 + r]) & 1ull) j |= 1u << r;
      // the kernel's terms
      int s2c = 0;
      for (int s = 0; s < op.nsh; ++s) s2c += __builtin_popcount(xt & (xt >> op.sh_d[s]) & op.sh_m[s]);
      int et = __builtin_popcount(xt & op.tmask) + 4 * s2c + phase;
      uint32_t B = 0;
      for (int r = 0; r < R; ++r)
        if (op.pq[r] != 0xFF && ((xt >> op.pq[r]) & 1u)) B |= 1u << r;
      bool keep = true;
      uint32_t wsum = 0;  // weights of phase slots on register qubits with j's bit set
      for (int i = 0; i < op.ncut; ++i) {
        const uint32_t q = op.cutq[i];
        const uint64_t l = (k >> op.cutm[i]) & 1ull;
        const bool reg = (regmask >> q) & 1u;
        const uint32_t bit = (uint32_t)((x >> q) & 1ull);
        if (!((op.cutz >> i) & 1u)) {
          if (bit != l) keep = false;
        } else if (l) {
          const uint32_t w = op.cutw[i];
          if (!reg) {
            et += (int)((w & 4u) ? 4 * bit : 0) + (int)((w & 1u) ? bit : 0) + (int)((w & 2u) ? 2 * bit : 0);
          } else {
            int r = 0;
            while (ord[8 + r] != (int)q) ++r;
            if (w & 4u) B ^= 1u << r;
            if (bit) wsum += (w & 3u);
          }
        }
      }
      const uint32_t field = (op.ereg[j / 8] >> (4 * (j % 8))) & 0xFu;
      int ek = (int)((field + (uint32_t)(et & 7)) & 7u);
      if (__builtin_popcount(B & j) & 1) ek = (ek + 4) & 7;
      ek = (ek + (int)wsum) & 7;
      bool kq;
      const int eq = (diag_exponent(op, x, k, kq) + phase) & 7;
      if (kq != keep || (keep && eq != ek)) {
        snprintf(buf, sizeof buf, "diag op %d at x=%llu: kernel e=%d keep=%d, qubit space e=%d keep=%d", oi,
                 (unsigned long long)x, ek, (int)keep, eq, (int)kq);
        return buf;
      }
      if (op.sign_only && keep && (eq & 3)) return "sign-only op with an exponent other than 0 or 4";
    }
  }
  // scale and phase: the factors the unscaled gates leave out
  const cd want = std::pow(cd(s2, 0), n_xy + n_h) * std::pow(cd(s2, s2), n_xy);  // |(1+i)/2| = 1/sqrt2, arg pi/4
  const cd have = (double)p.scale * omega(p.phase_e);
  if (std::abs(want - have) > 1e-6 * std::abs(want)) {
    snprintf(buf, sizeof buf, "pass factor: want %g%+gi, scale*w^e %g%+gi", want.real(), want.imag(), have.real(),
             have.imag());
    return buf;
  }
  return "";
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
      for (const Level& L : S.levels)
        for (const PassDesc& pd : L.passes)
          if (pd.k >= 8 && pd.low == 5 && !pd.general_gates && pd.op_count > 0) {
            const std::string e = check_register_pass(S, pd, k);
            if (!e.empty()) {
              printf("tables: half %d: %s\n", h, e.c_str());
              return 1;
            }
          }
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
