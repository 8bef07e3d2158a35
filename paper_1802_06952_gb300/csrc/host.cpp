// Host logic of libsim: random grid circuit generator, canonical gate-list text,
// cut planner (E_int, copy bits, half-circuits, copy tree) and the pass scheduler
// of the fused complex64 sweeps.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <set>
#include <sstream>
#include <stdexcept>
#include <tuple>

#include "sim_internal.h"

namespace sim {

// splitmix64 (Steele, Lea, Flood 2014), used for the X^1/2 / Y^1/2 draws and the
// amplitude selection.
uint64_t splitmix64_next(uint64_t& state) {
  state += 0x9E3779B97F4A7C15ull;
  uint64_t z = state;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

static const char* kGateName[] = {"H", "X2", "Y2", "T", "CZ", "CX", "X", "CT", "CY2"};
constexpr int kNumGateNames = 9;

// CZ couplers of pattern p (1..8) on an R x C grid whose cut lies above row b.
// Patterns 1-4: horizontal (r,c)-(r,c+1) with (r%2, c%2) = (0,0), (1,1), (0,1), (1,0).
// Patterns 5-8: vertical (r,c)-(r+1,c); 5/6 on rows of the other parity than b-1,
// 7/8 on rows of the same parity as b-1 (these hold the couplers crossing the
// cut); 5 and 7 take r+c even, 6 and 8 r+c odd.
static void couplers(int R, int C, int b, int p, std::vector<std::pair<int, int>>& out) {
  out.clear();
  if (p <= 4) {
    static const int want_r[4] = {0, 1, 0, 1};
    static const int want_c[4] = {0, 1, 1, 0};
    for (int r = 0; r < R; ++r)
      for (int c = 0; c + 1 < C; ++c)
        if (r % 2 == want_r[p - 1] && c % 2 == want_c[p - 1])
          out.emplace_back(r * C + c, r * C + c + 1);
  } else {
    const bool cut_parity = (p == 7 || p == 8);
    const bool even = (p == 5 || p == 7);
    const int bp = ((b - 1) % 2 + 2) % 2;
    for (int r = 0; r + 1 < R; ++r)
      for (int c = 0; c < C; ++c)
        if (((r % 2) == bp) == cut_parity && (((r + c) % 2) == 0) == even)
          out.emplace_back(r * C + c, (r + 1) * C + c);
  }
}

// Gate rule of the random circuits: layer 0 is H on all qubits; layer t >= 1 holds
// the CZs of pattern ((t-1) mod 8) + 1; for t >= 2 a qubit that was in a CZ at t-1
// and is not in one at t gets T if this is its first gate after H, else X^1/2 or
// Y^1/2 from one splitmix64 draw (top bit 1 -> Y^1/2), in (layer, qubit) order.
std::string generate_circuit(int R, int C, int depth, uint64_t seed, int cut_row, Circuit& out, int t_in_pool) {
  if (R < 1 || C < 1 || R * C > 64 || depth < 1) return "grid must have 1..64 qubits and depth >= 1";
  const int n = R * C;
  const int b = cut_row > 0 ? cut_row : R / 2;
  out = Circuit();
  out.R = R; out.C = C; out.depth = depth; out.seed = seed; out.cut_row = b; out.n = n;
  uint64_t rng = seed;
  std::vector<char> had_first(n, 0), prev(n, 0), cur(n, 0);
  std::vector<std::pair<int, int>> pairs;
  for (int t = 0; t < depth; ++t) {
    std::vector<Gate> layer;
    if (t == 0) {
      for (int q = 0; q < n; ++q) layer.push_back({0, G_H, q, -1});
    } else {
      couplers(R, C, b, ((t - 1) % 8) + 1, pairs);
      std::fill(cur.begin(), cur.end(), 0);
      for (auto& pr : pairs) {
        cur[pr.first] = cur[pr.second] = 1;
        layer.push_back({t, G_CZ, pr.first, pr.second});
      }
      if (t >= 2) {
        for (int q = 0; q < n; ++q) {
          if (prev[q] && !cur[q]) {
            if (!had_first[q]) {
              had_first[q] = 1;
              layer.push_back({t, G_T, q, -1});
            } else {
              uint64_t r = splitmix64_next(rng);
              if (t_in_pool) {
                // the T-in-pool variant: uniform over {X^1/2, Y^1/2, T}
                const uint64_t k3 = (r >> 32) % 3;
                layer.push_back({t, k3 == 0 ? G_X2 : (k3 == 1 ? G_Y2 : G_T), q, -1});
              } else {
                layer.push_back({t, (r >> 63) ? G_Y2 : G_X2, q, -1});
              }
            }
          }
        }
      }
      prev = cur;
    }
    std::sort(layer.begin(), layer.end(), [](const Gate& a, const Gate& b2) { return a.q1 < b2.q1; });
    out.gates.insert(out.gates.end(), layer.begin(), layer.end());
  }
  return "";
}

std::string circuit_text(const Circuit& c) {
  std::string s;
  char buf[96];
  snprintf(buf, sizeof buf, "circuit %d %d %d %llu\n", c.R, c.C, c.depth, (unsigned long long)c.seed);
  s += buf;
  for (const Gate& g : c.gates) {
    if (is_two_qubit(g.code))
      snprintf(buf, sizeof buf, "%d %s %d %d\n", g.t, kGateName[g.code], g.q1, g.q2);
    else
      snprintf(buf, sizeof buf, "%d %s %d\n", g.t, kGateName[g.code], g.q1);
    s += buf;
  }
  return s;
}

std::string parse_circuit(const char* text, Circuit& out) {
  out = Circuit();
  std::istringstream in(text);
  std::string line;
  bool have_head = false;
  int last_t = 0;
  std::vector<int> used_at;  // layer in which each qubit was last used
  while (std::getline(in, line)) {
    size_t a = line.find_first_not_of(" \t\r");
    if (a == std::string::npos || line[a] == '#') continue;
    std::istringstream ls(line);
    if (!have_head) {
      std::string kw;
      long long R, C, d;
      unsigned long long seed;
      if (!(ls >> kw >> R >> C >> d >> seed) || kw != "circuit") return "gate list must start with 'circuit R C depth seed'";
      if (R < 1 || C < 1 || R * C > 64 || d < 1) return "gate list header has a bad grid shape or depth";
      out.R = (int)R; out.C = (int)C; out.depth = (int)d; out.seed = seed; out.n = (int)(R * C);
      out.cut_row = out.R / 2;
      used_at.assign(out.n, -1);
      have_head = true;
      continue;
    }
    long long t, q1, q2 = -1;
    std::string nm;
    if (!(ls >> t >> nm >> q1)) return "malformed gate line: " + line;
    int code = -1;
    for (int i = 0; i < kNumGateNames; ++i)
      if (i != G_X && nm == kGateName[i]) code = i;
    if (code < 0) return "unknown gate name: " + nm;
    const bool two = is_two_qubit(code);
    if (two && !(ls >> q2)) return nm + " needs two qubits: " + line;
    if (t < 0 || t >= out.depth) return "gate layer out of range: " + line;
    if (t < last_t) return "gates must be ordered by layer";
    last_t = (int)t;
    if (q1 < 0 || q1 >= out.n || (two && (q2 < 0 || q2 >= out.n || q2 == q1)))
      return "qubit out of range: " + line;
    if (used_at[q1] == t || (two && used_at[q2] == t)) return "qubit used twice in one layer: " + line;
    used_at[q1] = (int)t;
    if (two) used_at[q2] = (int)t;
    Gate g{(int)t, code, (int)q1, (int)(two ? q2 : -1)};
    if (code == G_CZ && g.q2 < g.q1) std::swap(g.q1, g.q2);  // a controlled gate keeps (control, target)
    out.gates.push_back(g);
  }
  if (!have_head) return "empty gate list";
  return "";
}

// Amplitude selection: Floyd's algorithm over [0, 2^nq), one draw per step,
// t = next() mod (j + 1); result sorted ascending.  count >= 2^nq gives all.
void select_indices(int nq, uint64_t count, uint64_t& state, std::vector<uint64_t>& out) {
  out.clear();
  const uint64_t universe = nq >= 64 ? ~0ull : (1ull << nq);
  if (nq < 64 && count >= universe) {
    out.resize(universe);
    for (uint64_t i = 0; i < universe; ++i) out[i] = i;
    return;
  }
  std::set<uint64_t> chosen;
  for (uint64_t j = universe - count; j < universe; ++j) {
    uint64_t t = splitmix64_next(state) % (j + 1);
    if (chosen.count(t))
      chosen.insert(j);
    else
      chosen.insert(t);
    if (j == universe - 1) break;  // guards the wrap when universe == 2^64 - 1
  }
  out.assign(chosen.begin(), chosen.end());
}

// ---------------------------------------------------------------------------
// Cut plan and schedules
// ---------------------------------------------------------------------------
namespace {

// A diagonal cut slot on half-local qubit q for copy bit m: P_l (w = 0: the upper
// end of a cut CZ, or the control of a cut controlled gate in either half) or the
// phase w^{w l x_q} (w = 4: Z^l on the lower end of a cut CZ; 1: T^l on the target
// of a cut controlled T).
struct CutSlot {
  int q, m;
  int w;
};

// The U^l slot on the target q of a cut controlled gate (code G_CX, G_CT, G_CY2)
struct UCut {
  int q, m, code;
};

struct HalfGateLists {
  // per layer: non-diagonal gates (qubit, code), T qubits, CZ pairs, diagonal cut
  // slots, and U^l slots on the targets of cut controlled gates
  std::vector<std::vector<std::pair<int, int>>> nondiag;
  std::vector<uint32_t> tmask;
  std::vector<std::vector<std::pair<int, int>>> cz;
  std::vector<std::vector<CutSlot>> cuts;
  std::vector<std::vector<UCut>> ucuts;
};

void gate_matrix(int code, double m[8]) {
  const double s = 1.0 / std::sqrt(2.0);
  // row-major [m00, m01, m10, m11], each (re, im)
  switch (code) {
    case G_H: {
      double v[8] = {s, 0, s, 0, s, 0, -s, 0};
      memcpy(m, v, sizeof v);
      break;
    }
    case G_X2: {  // 1/2 [[1+i, 1-i], [1-i, 1+i]]
      double v[8] = {0.5, 0.5, 0.5, -0.5, 0.5, -0.5, 0.5, 0.5};
      memcpy(m, v, sizeof v);
      break;
    }
    case G_Y2: {  // 1/2 [[1+i, -1-i], [1+i, 1+i]]
      double v[8] = {0.5, 0.5, -0.5, -0.5, 0.5, 0.5, 0.5, 0.5};
      memcpy(m, v, sizeof v);
      break;
    }
    case G_X: {  // [[0, 1], [1, 0]]
      double v[8] = {0, 0, 1, 0, 1, 0, 0, 0};
      memcpy(m, v, sizeof v);
      break;
    }
    case G_T: {  // diag(1, (1+i)/sqrt2): the T^l slot of the plain path
      double v[8] = {1, 0, 0, 0, 0, 0, s, s};
      memcpy(m, v, sizeof v);
      break;
    }
    default: {
      double v[8] = {1, 0, 0, 0, 0, 0, 1, 0};
      memcpy(m, v, sizeof v);
    }
  }
}

OpRec make_gate(int code, int q, int cond = -1) {
  OpRec o;
  memset(&o, 0, sizeof o);
  o.type = OP_GATE;
  o.q = q;
  o.lq = -1;
  o.cond = cond;
  o.kind = code == G_X2 ? 1 : code == G_Y2 ? 2 : code == G_H ? 3 : code == G_X ? 4 : 0;
  gate_matrix(code, o.md);
  for (int i = 0; i < 8; ++i) o.m[i] = (float)o.md[i];
  return o;
}

// One or more DIAG ops for a layer: T mask, CZ pairs grouped by distance
// (x & (x >> d) & mask counts pairs (a, a + d) with both bits set), cut slots.
void make_diags(uint32_t tmask, const std::vector<std::pair<int, int>>& cz, const std::vector<CutSlot>& cuts,
                std::vector<OpRec>& out) {
  std::map<int, uint32_t> by_d;
  for (auto& p : cz) {
    int a = std::min(p.first, p.second), b = std::max(p.first, p.second);
    by_d[b - a] |= (1u << a);
  }
  std::vector<std::pair<int, uint32_t>> cls(by_d.begin(), by_d.end());
  size_t ci = 0, si = 0;
  bool first = true;
  while (first || ci < cls.size() || si < cuts.size()) {
    OpRec o;
    memset(&o, 0, sizeof o);
    o.type = OP_DIAG;
    o.lq = -1;
    o.q = -1;
    if (first) o.tmask = tmask;
    first = false;
    while (ci < cls.size() && o.nsh < kMaxShift) {
      o.sh_d[o.nsh] = (uint32_t)cls[ci].first;
      o.sh_m[o.nsh] = cls[ci].second;
      ++o.nsh;
      ++ci;
    }
    while (si < cuts.size() && o.ncut < kMaxCutSlots) {
      o.cutq[o.ncut] = (uint8_t)cuts[si].q;
      o.cutm[o.ncut] = (uint8_t)cuts[si].m;
      if (cuts[si].w) {
        o.cutz |= 1u << o.ncut;
        o.cutw[o.ncut] = (uint8_t)(cuts[si].w & 7);
      }
      ++o.ncut;
      ++si;
    }
    if (o.tmask || o.nsh || o.ncut) out.push_back(o);
  }
}

// An item of a level's op sequence before the passes are formed: a non-diagonal
// gate, or the diagonal terms of one layer (T qubits, CZ pairs, cut slots), kept
// apart so that a pass can apply the terms on some qubits and leave the others.
struct SeqItem {
  bool is_gate = false;
  OpRec gate;
  uint32_t tmask = 0;
  std::vector<std::pair<int, int>> cz;
  std::vector<CutSlot> cuts;
  bool empty_diag() const { return !is_gate && tmask == 0 && cz.empty() && cuts.empty(); }
};

SeqItem gate_item(const OpRec& o) {
  SeqItem it;
  it.is_gate = true;
  it.gate = o;
  return it;
}

SeqItem diag_item(uint32_t tmask, const std::vector<std::pair<int, int>>& cz, const std::vector<CutSlot>& cuts) {
  SeqItem it;
  it.tmask = tmask;
  it.cz = cz;
  it.cuts = cuts;
  return it;
}

// Pass formation (Section 2.2's n_i fused passes, Section 2.4's combined diagonals).
// Each pass stages k local qubits: the low `low` bits (coalesced rows) and the
// qubits of the gates it applies, in sequence order.  The scan runs over the whole
// remaining sequence: a gate whose qubit no longer fits is left for a later pass
// and its qubit is blocked, and so is every later item that touches a blocked
// qubit (a diagonal term on a blocked qubit blocks all of its qubits), so that
// everything a pass applies comes after everything it depends on.  Diagonal terms
// need no staged qubit (their phase depends on the full index), so every term on
// unblocked qubits is applied where the scan meets it.  Items left over keep their
// order for the next pass.  With k < n at most k - 1 low bits are reserved, so
// every pass applies at least the item it starts with.  In order (in_order), a
// pass instead ends at the first gate that does not fit.
std::vector<std::vector<OpRec>> form_passes(int k, int low, std::vector<SeqItem> items, bool in_order) {
  std::vector<std::vector<OpRec>> out;
  const uint32_t low_mask = (1u << low) - 1;
  while (!items.empty()) {
    uint32_t staged = low_mask, blocked = 0;
    int cnt = low;
    bool full = false;
    std::vector<OpRec> pass;
    std::vector<SeqItem> rest;
    // Applied diagonal terms are held back and merged into one diagonal op until a
    // gate touches one of their qubits or a new term shares a qubit with them
    // (diagonal terms commute with each other and with gates on other qubits).
    SeqItem pend;
    uint32_t pend_q = 0;
    auto flush = [&]() {
      if (pend_q) make_diags(pend.tmask, pend.cz, pend.cuts, pass);
      pend = SeqItem();
      pend_q = 0;
    };
    for (const SeqItem& it : items) {
      if (full) {
        rest.push_back(it);
        continue;
      }
      if (it.is_gate) {
        const uint32_t b = 1u << it.gate.q;
        if (!(blocked & b) && ((staged & b) || cnt < k)) {
          if (!(staged & b)) {
            staged |= b;
            ++cnt;
          }
          if (pend_q & b) flush();
          pass.push_back(it.gate);
        } else {
          blocked |= b;
          rest.push_back(it);
          if (in_order) full = true;  // the pass ends here
        }
      } else {
        // the terms of one layer act on distinct qubits: each is applied or left
        SeqItem now, later;
        now.tmask = it.tmask & ~blocked;
        later.tmask = it.tmask & blocked;
        for (const auto& pr : it.cz)
          ((blocked >> pr.first) & 1u || (blocked >> pr.second) & 1u ? later.cz : now.cz).push_back(pr);
        for (const CutSlot& sl : it.cuts) ((blocked >> sl.q) & 1u ? later.cuts : now.cuts).push_back(sl);
        for (const auto& pr : later.cz) blocked |= (1u << pr.first) | (1u << pr.second);
        if (!now.empty_diag()) {
          uint32_t q = now.tmask;
          for (const auto& pr : now.cz) q |= (1u << pr.first) | (1u << pr.second);
          for (const CutSlot& sl : now.cuts) q |= 1u << sl.q;
          if (pend_q & q) flush();
          pend.tmask |= now.tmask;
          pend.cz.insert(pend.cz.end(), now.cz.begin(), now.cz.end());
          pend.cuts.insert(pend.cuts.end(), now.cuts.begin(), now.cuts.end());
          pend_q |= q;
        }
        if (!later.empty_diag()) rest.push_back(later);
      }
      // room for the exchanges of the register-blocked sweep
      if ((int)pass.size() >= kMaxPassOps - 24) full = true;
    }
    flush();
    if (pass.empty()) throw std::logic_error("pass formation made no progress");
    out.push_back(std::move(pass));
    items.swap(rest);
  }
  return out;
}

// Number of fused passes a level's sequence forms into.
int count_passes(int n, int kmax, const std::vector<SeqItem>& items, bool in_order) {
  if (items.empty()) return 1;
  const int k = std::min(n, kmax);
  const int low = k < n ? std::min(5, k - 1) : std::min(5, k);
  return (int)form_passes(k, low, items, in_order).size();
}

// Ops of a child level that commute with everything the child must keep are
// applied once per parent node instead of once per child (the shared prefixes of
// Section 2.3.2, extended by commutation).  The child keeps its cut slots (the
// copy-dependent items; all diagonal) and every op that does not commute past what
// it keeps: a non-diagonal gate on a qubit a kept item touches, or a diagonal term
// on a qubit a kept non-diagonal gate touches.  Hoisted ops keep their order and
// follow the parent's own ops.  The move is made only if the passes it costs do not
// outweigh those it saves, at 2^bits children per parent.
void hoist_into_parent(int n, int kmax, bool in_order, std::vector<SeqItem>& parent, std::vector<SeqItem>& child,
                       int bits) {
  uint32_t kept_diag = 0, kept_gate = 0;  // qubits touched by kept diagonal terms / kept gates
  std::vector<SeqItem> up, keep;
  for (const SeqItem& it : child) {
    if (it.is_gate) {
      const uint32_t b = 1u << it.gate.q;
      if ((kept_diag | kept_gate) & b) {
        keep.push_back(it);
        kept_gate |= b;
      } else {
        up.push_back(it);
      }
      continue;
    }
    SeqItem u, st;
    st.cuts = it.cuts;
    for (int q = 0; q < 32; ++q)
      if ((it.tmask >> q) & 1u) ((kept_gate >> q) & 1u ? st.tmask : u.tmask) |= 1u << q;
    for (const auto& pr : it.cz)
      ((kept_gate >> pr.first) & 1u || (kept_gate >> pr.second) & 1u ? st.cz : u.cz).push_back(pr);
    kept_diag |= st.tmask;
    for (const auto& pr : st.cz) kept_diag |= (1u << pr.first) | (1u << pr.second);
    for (const CutSlot& sl : st.cuts) kept_diag |= 1u << sl.q;
    if (!u.empty_diag()) up.push_back(u);
    if (!st.empty_diag()) keep.push_back(st);
  }
  if (up.empty()) return;
  std::vector<SeqItem> parent2 = parent;
  parent2.insert(parent2.end(), up.begin(), up.end());
  const int64_t w = (int64_t)1 << std::min(bits, 40);
  const int64_t before = count_passes(n, kmax, parent, in_order) + w * count_passes(n, kmax, child, in_order);
  const int64_t after = count_passes(n, kmax, parent2, in_order) + w * count_passes(n, kmax, keep, in_order);
  if (after > before) return;
  parent.swap(parent2);
  child.swap(keep);
}

// The passes of one copy-tree level: formed as above, then each given its rank
// order (which staged qubit sits on which lane, warp and register bit).
void split_passes(int n, int kmax, const std::vector<SeqItem>& items, int first_src, bool in_order,
                  std::vector<PassDesc>& passes, std::vector<OpRec>& ops) {
  const int k = std::min(n, kmax);
  const int low = k < n ? std::min(5, k - 1) : std::min(5, k);
  const uint32_t low_mask = (1u << low) - 1;
  bool first = true;
  if (items.empty()) {
    PassDesc p;
    memset(&p, 0, sizeof p);
    p.k = k;
    p.low = low;
    p.local_mask = (k >= 32 ? 0xFFFFFFFFu : ((1u << k) - 1));
    p.op_begin = (int)ops.size();
    p.op_count = 0;
    p.src = first_src;
    p.scale = 1.f;
    p.phase_e = 0;
    p.phase_op = -1;
    for (int r = 0; r < k; ++r) p.order[r] = (uint8_t)r;
    passes.push_back(p);
    return;
  }
  for (const std::vector<OpRec>& seq : form_passes(k, low, items, in_order)) {
    const size_t i = 0, j = seq.size();
    uint32_t local = low_mask;
    int cnt = low;
    for (const OpRec& o : seq)
      if (o.type == OP_GATE && !(local & (1u << o.q))) {
        local |= 1u << o.q;
        ++cnt;
      }
    if (cnt > k) throw std::logic_error("pass stages more than k qubits");
    // fill the remaining local slots with the lowest unused qubits
    for (int q = 0; q < n && cnt < k; ++q)
      if (!(local & (1u << q))) { local |= 1u << q; ++cnt; }
    PassDesc p;
    memset(&p, 0, sizeof p);
    p.k = k;
    p.low = low;
    p.local_mask = local;
    p.op_begin = (int)ops.size();
    p.op_count = (int)(j - i);
    p.src = first ? first_src : SRC_SELF;
    // rank order: the low bits first; then (k >= 8) three warp-bit ranks and k-8
    // register-bit ranks; the qubits with the most gates in the pass take the
    // register ranks, qubits without gates the warp ranks
    int gates_on[32] = {0};
    for (size_t t = i; t < j; ++t)
      if (seq[t].type == OP_GATE) ++gates_on[seq[t].q];
    std::vector<int> hi;
    for (int q = low; q < n; ++q)
      if (local & (1u << q)) hi.push_back(q);
    std::stable_sort(hi.begin(), hi.end(), [&](int a, int b2) { return gates_on[a] > gates_on[b2]; });
    const int nreg = k >= 8 ? k - 8 : 0;
    int r = 0;
    if (k >= 8 && low == 5) {
      // storage order: qubits 0..4, then the other local qubits ascending
      for (int q = 0; q < 5; ++q) p.sorder[r++] = (uint8_t)q;
      std::vector<int> rest_s;
      for (int q = 5; q < n; ++q)
        if (local & (1u << q)) rest_s.push_back(q);
      for (int q : rest_s) p.sorder[r++] = (uint8_t)q;
      // compute order: the 5 + nreg local qubits with the most gates take the lane
      // and register ranks (ties: qubits 0..4 first, so that no transpose is needed
      // when the low qubits are as busy), the rest the three warp ranks
      std::vector<int> all;
      for (int q = 0; q < n; ++q)
        if (local & (1u << q)) all.push_back(q);
      std::stable_sort(all.begin(), all.end(), [&](int a, int b2) {
        if (gates_on[a] != gates_on[b2]) return gates_on[a] > gates_on[b2];
        return a < b2;
      });
      if (nreg >= 2) {
        // 256-bit runs: register ranks 8, 9 = qubits 0, 1; lanes 0..2 = qubits 2..4,
        // so that 8 lanes read 256 contiguous bytes; the busiest other qubits take the
        // remaining register ranks, the next two lanes 3 and 4, the rest the warp
        // ranks; loads and stores use this order directly
        std::vector<int> rest;
        for (int q : all)
          if (q > 4) rest.push_back(q);
        std::vector<int> regs2(rest.begin(), rest.begin() + (nreg - 2));
        std::vector<int> lanes2 = {2, 3, 4};
        lanes2.insert(lanes2.end(), rest.begin() + (nreg - 2), rest.begin() + nreg);
        std::vector<int> warps2(rest.begin() + nreg, rest.end());
        std::sort(warps2.begin(), warps2.end());
        r = 0;
        for (int q : lanes2) p.order[r++] = (uint8_t)q;
        for (int q : warps2) p.order[r++] = (uint8_t)q;
        p.order[r++] = 0;
        p.order[r++] = 1;
        for (int q : regs2) p.order[r++] = (uint8_t)q;
        for (int t2 = 0; t2 < k; ++t2) p.sorder[t2] = p.order[t2];
        memset(p.swz, 0, sizeof p.swz);
        p.transpose = 0;
        p.vec4 = 1;
      } else {
      std::vector<int> lanes(all.begin(), all.begin() + 5);
      std::vector<int> regs(all.begin() + 5, all.begin() + 5 + nreg);
      std::vector<int> warps(all.begin() + 5 + nreg, all.end());
      // keep a low qubit on the lane rank equal to its storage rank when it is a lane
      std::vector<int> lane_slot(5, -1);
      for (int q : lanes)
        if (q < 5) lane_slot[q] = q;
      size_t li = 0;
      for (int s = 0; s < 5; ++s) {
        if (lane_slot[s] >= 0) continue;
        while (lanes[li] < 5) ++li;
        lane_slot[s] = lanes[li++];
      }
      std::sort(warps.begin(), warps.end());
      r = 0;
      for (int s = 0; s < 5; ++s) p.order[r++] = (uint8_t)lane_slot[s];
      for (int q : warps) p.order[r++] = (uint8_t)q;
      for (int q : regs) p.order[r++] = (uint8_t)q;
      p.transpose = 0;
      for (int t2 = 0; t2 < k; ++t2)
        if (p.order[t2] != p.sorder[t2]) p.transpose = 1;
      // swizzle: the compute lanes, read at their storage ranks, must reach all 16
      // low slots of shared memory (two lanes per 8-byte bank pair): storage ranks
      // 0..3 cover their own low bits; each compute lane at a storage rank >= 4 adds
      // one low bit not yet covered
      int srank_of[32];
      for (int t2 = 0; t2 < 32; ++t2) srank_of[t2] = -1;
      for (int t2 = 0; t2 < k; ++t2) srank_of[p.sorder[t2]] = t2;
      unsigned covered = 0;
      for (int s = 0; s < 5; ++s) {
        const int sr = srank_of[p.order[s]];
        if (sr < 4) covered |= 1u << sr;
      }
      for (int s = 0; s < 5; ++s) {
        const int sr = srank_of[p.order[s]];
        if (sr < 4) continue;
        for (int b = 0; b < 4; ++b)
          if (!(covered & (1u << b))) {
            p.swz[sr] = (uint8_t)(1u << b);
            covered |= 1u << b;
            break;
          }
      }
      }
    } else {
      for (int q = 0; q < low; ++q) p.order[r++] = (uint8_t)q;
      // warp ranks: the qubits after the first nreg (fewest gates), lowest first
      std::vector<int> warp_q(hi.begin() + nreg, hi.end());
      std::sort(warp_q.begin(), warp_q.end());
      for (int q : warp_q) p.order[r++] = (uint8_t)q;
      for (int t2 = 0; t2 < nreg; ++t2) p.order[r++] = (uint8_t)hi[t2];
      for (int t2 = 0; t2 < k; ++t2) p.sorder[t2] = p.order[t2];
    }
    // Ops of the pass with the rank map at each op.  Register-blocked passes with
    // 256-bit runs (vec4) exchange warp ranks 5+m with register ranks 10+m
    // (m < nsw) when a gate hits one of those warp ranks, which turns the
    // exchanged warp qubits into register qubits (one shared-memory round trip,
    // the cost of one warp-rank gate, for every later gate on them).
    const int R = (k >= 8 && low == 5) ? k - 8 : 0;
    // (measured: a gain with three register ranks to exchange, k = 13; a loss with
    // one or two, where fewer gates move per exchange)
    const int nsw = (p.vec4 && R >= 5) ? 3 : 0;
    int ord[16];
    int rank_of[32], rank0[32];
    for (int t2 = 0; t2 < 32; ++t2) rank_of[t2] = rank0[t2] = -1;
    for (int t2 = 0; t2 < 16; ++t2) ord[t2] = t2 < k ? p.order[t2] : -1;
    for (int t2 = 0; t2 < k; ++t2) rank_of[p.order[t2]] = rank0[p.order[t2]] = t2;
    p.warp_gates = 0;
    p.general_gates = 0;
    int n_xy = 0, n_h = 0;
    p.phase_op = -1;
    auto fill_diag_tables = [&](OpRec& o) {
      uint32_t regmask = 0;
      for (int t2 = 0; t2 < R; ++t2) regmask |= 1u << ord[8 + t2];
      o.regmask = regmask;
      memset(o.rq, 0xFF, sizeof o.rq);
      for (int t2 = 0; t2 < R; ++t2) o.rq[t2] = (uint8_t)ord[8 + t2];
      memset(o.ereg, 0, sizeof o.ereg);
      for (int jj = 0; jj < (1 << R); ++jj) {
        uint32_t xr = 0;
        for (int t2 = 0; t2 < R; ++t2)
          if ((jj >> t2) & 1) xr |= 1u << ord[8 + t2];
        int s2 = 0;
        for (int sc = 0; sc < o.nsh; ++sc) s2 += __builtin_popcount(xr & (xr >> o.sh_d[sc]) & o.sh_m[sc]);
        const int e = (__builtin_popcount(xr & o.tmask) + 4 * s2) & 7;
        o.ereg[jj / 8] |= (uint32_t)e << (4 * (jj % 8));
      }
      for (int t2 = 0; t2 < 8; ++t2) o.pq[t2] = 0xFF;
      for (int t2 = 0; t2 < R; ++t2) {
        const int q = ord[8 + t2];
        for (int sc = 0; sc < o.nsh; ++sc) {
          const int d = (int)o.sh_d[sc];
          int partner = -1;
          if ((o.sh_m[sc] >> q) & 1u) partner = q + d;                      // pair (q, q + d)
          if (q - d >= 0 && ((o.sh_m[sc] >> (q - d)) & 1u)) partner = q - d;  // pair (q - d, q)
          if (partner >= 0 && !((regmask >> partner) & 1u)) o.pq[t2] = (uint8_t)partner;
        }
      }
    };
    for (size_t t = i; t < j; ++t) {
      OpRec o = seq[t];
      if (o.type == OP_GATE) {
        const int cur = rank_of[o.q];
        // exchange only when the rest of the pass has clearly more gates on the
        // qubits coming in (the warp ranks) than on those going out (which would
        // bring them back): each exchange costs about one warp-rank gate
        int in_cnt = 0, out_cnt = 0;
        if (nsw > 0 && cur >= 5 && cur < 5 + nsw)
          for (size_t u = t; u < j; ++u) {
            if (seq[u].type != OP_GATE) continue;
            const int ru = rank_of[seq[u].q];
            if (ru >= 5 && ru < 5 + nsw) ++in_cnt;
            if (ru >= 10 && ru < 10 + nsw) ++out_cnt;
          }
        if (nsw > 0 && cur >= 5 && cur < 5 + nsw && in_cnt >= out_cnt + 2) {
          OpRec sw;
          memset(&sw, 0, sizeof sw);
          sw.type = OP_SWAP;
          for (int m = 0; m < nsw; ++m) std::swap(ord[5 + m], ord[10 + m]);
          for (int t2 = 0; t2 < k; ++t2) rank_of[ord[t2]] = t2;
          for (int t2 = 0; t2 < 8; ++t2) sw.tq[t2] = (uint8_t)ord[t2];
          ops.push_back(sw);
          ++p.warp_gates;  // needs the shared-memory slots
        }
        o.lq = rank_of[o.q];
        o.lq0 = rank0[o.q];
        if (k >= 8 && o.lq >= 5 && o.lq < 8) ++p.warp_gates;
        if (o.kind == 1 || o.kind == 2)
          ++n_xy;
        else if (o.kind == 3)
          ++n_h;
        else
          ++p.general_gates;
      } else {
        if (R > 0) fill_diag_tables(o);
        // exponents all 0 or 4 (CZ terms, Z^l and P_l slots only): a sign flip
        bool sign_only = o.tmask == 0;
        for (int i = 0; i < o.ncut; ++i)
          if (((o.cutz >> i) & 1u) && o.cutw[i] != 4) sign_only = false;
        o.sign_only = sign_only ? 1 : 0;
        // the pass's phase w^(n_xy) goes into the last op that takes general
        // phases anyway, so that the sign-only ops stay sign-only
        if (!sign_only) p.phase_op = (int)(ops.size() - (size_t)p.op_begin);
      }
      ops.push_back(o);
    }
    p.op_count = (int)(ops.size() - (size_t)p.op_begin);
    // stores use the map after the last exchange
    if (p.vec4)
      for (int t2 = 0; t2 < k; ++t2) p.sorder[t2] = (uint8_t)ord[t2];
    p.scale = (float)std::ldexp(n_xy + n_h == 0 ? 1.0 : ((n_xy + n_h) & 1 ? 0.70710678118654752440 : 1.0),
                                -((n_xy + n_h) / 2));
    p.phase_e = n_xy & 7;
    // without such an op the store applies the phase; w^4 = -1 is the scale's sign
    if (p.phase_op < 0 && p.phase_e == 4) {
      p.scale = -p.scale;
      p.phase_e = 0;
    }
    passes.push_back(p);
    first = false;
  }
}

// The fused schedule and the plain layers of one half-circuit (or one part of a
// multi-part cut) from its gate lists: branch[j] is the j-th layer holding its cut
// slots, branch_bits[j] the number of copy bits those slots fix (its copy bits are
// numbered by layer, so each level fixes the next ones).
void build_half(const Circuit& c, const HalfGateLists& H, int n, const std::vector<int>& branch,
                const std::vector<int>& branch_bits, int fuse, bool in_order, HalfSchedule& S,
                std::vector<PlainLayer>& plain_layers) {
  S.n = n;
  // plain pass count (Section 2.4): one per non-diagonal gate, one per layer
  // holding any diagonal gate (T, CZ, or cut slot)
  int plain = 0;
  for (int t = 0; t < c.depth; ++t) {
    plain += (int)H.nondiag[t].size() + (int)H.ucuts[t].size();
    if (H.tmask[t] || !H.cz[t].empty() || !H.cuts[t].empty()) ++plain;
  }
  S.plain_passes = plain;
  // does layer 0 put H on every qubit of the half?
  bool uniform = c.depth > 0 && (int)H.nondiag[0].size() == n && H.tmask[0] == 0 &&
                 H.cz[0].empty() && H.cuts[0].empty();
  if (uniform)
    for (auto& p : H.nondiag[0])
      if (p.second != G_H) uniform = false;

  const int nlev = (int)branch.size() + 1;
  int bits = 0;
  std::vector<std::vector<SeqItem>> seqs;
  for (int j = 0; j < nlev; ++j) {
    Level L;
    L.branch_layer = j == 0 ? -1 : branch[j - 1];
    L.bits_before = bits;
    bits += j > 0 ? branch_bits[j - 1] : 0;
    L.bits_total = bits;
    const int t_begin = j == 0 ? 0 : branch[j - 1];
    const int t_end = j + 1 < nlev ? branch[j] : c.depth - 1;  // inclusive
    std::vector<SeqItem> seq;
    for (int t = t_begin; t <= t_end; ++t) {
      const bool own_cut_layer = (j > 0 && t == t_begin);
      if (own_cut_layer) {
        // this level applies only the cut slots of its branch layer here.  A U^l
        // slot is written as copy-independent gates around one diagonal phase slot
        // w^{b l x_q}, so the fused passes need no copy-dependent gate:
        //   X^l        = H Z^l H                       (H Z H = X, H H = I; b = 4)
        //   T^l        = diag(1, w^l)                  (b = 1)
        //   (Y^1/2)^l  = X^1/2 X^1/2 X^1/2 S^l X^1/2   (X^-1/2 S X^1/2 = Y^1/2 and
        //                (X^1/2)^4 = I; b = 2), gates listed in time order below
        // Their common factors are the same in every copy.  The slots act on qubits
        // no other gate of the layer touches.
        std::vector<CutSlot> slots = H.cuts[t];
        for (const UCut& u : H.ucuts[t]) {
          if (u.code == G_CX) seq.push_back(gate_item(make_gate(G_H, u.q)));
          if (u.code == G_CY2) seq.push_back(gate_item(make_gate(G_X2, u.q)));
          slots.push_back({u.q, u.m, u.code == G_CX ? 4 : u.code == G_CT ? 1 : 2});
        }
        seq.push_back(diag_item(0, {}, slots));
        for (const UCut& u : H.ucuts[t]) {
          if (u.code == G_CX) seq.push_back(gate_item(make_gate(G_H, u.q)));
          if (u.code == G_CY2)
            for (int r = 0; r < 3; ++r) seq.push_back(gate_item(make_gate(G_X2, u.q)));
        }
        continue;
      }
      if (!(j == 0 && t == 0 && uniform))
        for (auto& p : H.nondiag[t]) seq.push_back(gate_item(make_gate(p.second, p.first)));
      const bool next_branch = (j + 1 < nlev && t == t_end);
      SeqItem d = diag_item(H.tmask[t], H.cz[t], next_branch ? std::vector<CutSlot>() : H.cuts[t]);
      if (!d.empty_diag()) seq.push_back(d);
    }
    S.levels.push_back(L);
    seqs.push_back(std::move(seq));
  }
  // copy-independent ops move up the tree where that saves work (bottom-up, so
  // that an op can climb several levels)
  for (int j = nlev - 1; j >= 1; --j) hoist_into_parent(n, fuse, in_order, seqs[j - 1], seqs[j], branch_bits[j - 1]);
  for (int j = 0; j < nlev; ++j) {
    const int first_src = j == 0 ? (uniform ? SRC_UNIFORM : SRC_ZERO) : SRC_PARENT;
    split_passes(n, fuse, seqs[j], first_src, in_order, S.levels[j].passes, S.ops);
  }

  // plain complex128 path: per layer, one op per non-diagonal gate, then the
  // combined diagonal of the layer with this copy's cut slots
  plain_layers.assign(c.depth, PlainLayer());
  for (int t = 0; t < c.depth; ++t) {
    for (auto& p : H.nondiag[t]) plain_layers[t].gates.push_back(make_gate(p.second, p.first));
    // the plain path applies U on the target in the copies with l_m = 1
    for (const UCut& u : H.ucuts[t])
      plain_layers[t].gates.push_back(
          make_gate(u.code == G_CX ? G_X : u.code == G_CT ? G_T : G_Y2, u.q, u.m));
    make_diags(H.tmask[t], H.cz[t], H.cuts[t], plain_layers[t].diags);
  }
}

}  // namespace

std::string build_cut_plan(const Circuit& c, int cut_row, int fuse_qubits, CutPlan& plan, int pass_order,
                           bool out_phase_cuts) {
  const int b = cut_row > 0 ? cut_row : c.R / 2;
  if (b < 1 || b >= c.R) return "cut row must lie strictly inside the grid";
  plan = CutPlan();
  plan.circ = c;
  plan.n_u = b * c.C;
  plan.n_l = c.n - plan.n_u;
  if (plan.n_u > 32 || plan.n_l > 32) return "each half must have at most 32 qubits";
  plan.fuse_qubits = fuse_qubits > 0 ? fuse_qubits : 13;
  if (plan.fuse_qubits < 4 || plan.fuse_qubits > 13) return "fuse_qubits must be in 4..13";
  if (pass_order < 0 || pass_order > 1) return "pass_order must be 0 or 1";
  plan.pass_order = pass_order;
  const int nu = plan.n_u;
  // Output-phase cuts (when asked for): a cut CZ at layer t with no non-diagonal
  // gate on either of its qubits after t commutes with every later gate, so it can
  // be applied to the final amplitudes as the sign (-1)^{x_h x_k} instead of being
  // split into copies.
  plan.out_phase_cuts = out_phase_cuts;
  std::vector<int> last_nondiag(c.n, -1);  // last layer with a non-diagonal gate on a qubit
  for (const Gate& g : c.gates)
    if (g.code != G_T && g.code != G_CZ) {
      last_nondiag[g.q1] = std::max(last_nondiag[g.q1], g.t);
      if (g.q2 >= 0) last_nondiag[g.q2] = std::max(last_nondiag[g.q2], g.t);
    }
  std::set<std::pair<int, int>> out_keys;  // (layer, upper qubit) of the output-phase cuts
  // E_int: CZs (and controlled X gates) with one endpoint in each half, numbered by
  // (layer, upper qubit)
  for (const Gate& g : c.gates) {
    if (g.code == G_CZ && g.q1 < nu && g.q2 >= nu) {
      // (at most 32: the output-sign codes are 32-bit; further ones stay copy bits)
      if (out_phase_cuts && plan.out_cz.size() < 32 && last_nondiag[g.q1] < g.t && last_nondiag[g.q2] < g.t) {
        plan.out_cz.emplace_back(g.q1, g.q2);
        out_keys.insert({g.t, g.q1});
        continue;
      }
      plan.cuts.push_back({g.t, g.q1, g.q2, 0});
    }
    if (is_controlled_u(g.code)) {
      const int a = std::min(g.q1, g.q2), b2 = std::max(g.q1, g.q2);
      if (!(a < nu && b2 >= nu))
        return std::string("a controlled gate (") + kGateName[g.code] +
               ") inside one half is not supported (only across the cut)";
      plan.cuts.push_back({g.t, a, b2, g.q1 < nu ? 1 : 2, g.code});
    }
  }
  std::sort(plan.cuts.begin(), plan.cuts.end(), [](const CutCZ& a, const CutCZ& b2) {
    return a.t != b2.t ? a.t < b2.t : a.h < b2.h;
  });
  plan.c = (int)plan.cuts.size();
  if (plan.c > 40) return "more than 40 cut CZs";
  std::map<std::pair<int, int>, int> cut_index;
  for (int m = 0; m < plan.c; ++m) cut_index[{plan.cuts[m].t, plan.cuts[m].h}] = m;

  HalfGateLists hl[2];
  for (int h = 0; h < 2; ++h) {
    hl[h].nondiag.assign(c.depth, {});
    hl[h].tmask.assign(c.depth, 0);
    hl[h].cz.assign(c.depth, {});
    hl[h].cuts.assign(c.depth, {});
    hl[h].ucuts.assign(c.depth, {});
  }
  for (const Gate& g : c.gates) {
    if (g.code == G_CZ) {
      if (g.q2 < nu) {
        hl[0].cz[g.t].emplace_back(g.q1, g.q2);
      } else if (g.q1 >= nu) {
        hl[1].cz[g.t].emplace_back(g.q1 - nu, g.q2 - nu);
      } else if (!out_keys.count({g.t, g.q1})) {
        int m = cut_index[{g.t, g.q1}];
        hl[0].cuts[g.t].push_back({g.q1, m, 0});
        hl[1].cuts[g.t].push_back({g.q2 - nu, m, 4});
      }
    } else if (is_controlled_u(g.code)) {
      const int a = std::min(g.q1, g.q2);
      const int m = cut_index[{g.t, a}];
      const int hc = g.q1 < nu ? 0 : 1;  // half of the control
      hl[hc].cuts[g.t].push_back({hc ? g.q1 - nu : g.q1, m, 0});
      hl[1 - hc].ucuts[g.t].push_back({hc ? g.q2 : g.q2 - nu, m, g.code});
    } else {
      int h = g.q1 < nu ? 0 : 1;
      int q = h ? g.q1 - nu : g.q1;
      if (g.code == G_T)
        hl[h].tmask[g.t] |= 1u << q;
      else
        hl[h].nondiag[g.t].emplace_back(q, g.code);
    }
  }
  // branch layers: distinct layers holding cuts, in order
  std::vector<int> branch;
  for (const CutCZ& x : plan.cuts)
    if (branch.empty() || branch.back() != x.t) branch.push_back(x.t);

  std::vector<int> branch_bits;
  for (int t : branch) {
    int nb = 0;
    for (const CutCZ& x : plan.cuts)
      if (x.t == t) ++nb;
    branch_bits.push_back(nb);
  }
  for (int h = 0; h < 2; ++h)
    build_half(c, hl[h], h ? plan.n_l : plan.n_u, branch, branch_bits, plan.fuse_qubits, plan.pass_order == 1,
               plan.sched[h], plan.plain[h]);
  return "";
}

std::string build_multi_plan(const Circuit& c, const std::vector<int>& cut_rows, int fuse_qubits, int pass_order,
                             MultiPlan& mp) {
  mp = MultiPlan();
  mp.circ = c;
  std::vector<int> rows = {0};
  for (int r : cut_rows) rows.push_back(r);
  rows.push_back(c.R);
  for (size_t i = 0; i + 1 < rows.size(); ++i)
    if (rows[i] >= rows[i + 1]) return "cut rows must increase strictly inside the grid";
  const int fuse = fuse_qubits > 0 ? fuse_qubits : 13;
  if (fuse < 4 || fuse > 13) return "fuse_qubits must be in 4..13";
  if (pass_order < 0 || pass_order > 1) return "pass_order must be 0 or 1";
  mp.t = (int)rows.size() - 1;
  std::vector<int> part_of(c.n, 0);
  for (int p = 0; p < mp.t; ++p) {
    mp.offset.push_back(rows[p] * c.C);
    mp.nq.push_back((rows[p + 1] - rows[p]) * c.C);
    if (mp.nq.back() > 32) return "a part has more than 32 qubits";
    for (int q = rows[p] * c.C; q < rows[p + 1] * c.C; ++q) part_of[q] = p;
  }
  // cut CZs per boundary, numbered by (layer, upper qubit)
  std::vector<std::vector<CutCZ>> cuts(mp.t);
  for (const Gate& g : c.gates) {
    if (is_controlled_u(g.code) || g.code == G_X) return "multi-part cuts take H, X^1/2, Y^1/2, T and CZ gates only";
    if (g.code != G_CZ) continue;
    const int pa = part_of[g.q1], pb = part_of[g.q2];  // q1 < q2
    if (pb - pa > 1) return "a CZ crosses more than one boundary";
    if (pb != pa) cuts[pb].push_back({g.t, g.q1, g.q2, 0});
  }
  mp.c.assign(mp.t, 0);
  std::map<std::pair<int, int>, std::pair<int, int>> where;  // (layer, upper qubit) -> (boundary, bit)
  for (int j = 1; j < mp.t; ++j) {
    std::sort(cuts[j].begin(), cuts[j].end(),
              [](const CutCZ& a, const CutCZ& b2) { return a.t != b2.t ? a.t < b2.t : a.h < b2.h; });
    mp.c[j] = (int)cuts[j].size();
    for (int i = 0; i < mp.c[j]; ++i) where[{cuts[j][i].t, cuts[j][i].h}] = {j, i};
  }
  // each part's slots in (layer, upper qubit) order -> its local copy bits
  mp.slot_bits.assign(mp.t, {});
  std::vector<std::map<std::pair<int, int>, int>> local(mp.t);  // (boundary, bit) -> local bit
  for (int p = 0; p < mp.t; ++p) {
    std::vector<std::tuple<int, int, int, int>> sl;  // (layer, upper qubit, boundary, bit)
    if (p > 0)
      for (int i = 0; i < mp.c[p]; ++i) sl.emplace_back(cuts[p][i].t, cuts[p][i].h, p, i);
    if (p + 1 < mp.t)
      for (int i = 0; i < mp.c[p + 1]; ++i) sl.emplace_back(cuts[p + 1][i].t, cuts[p + 1][i].h, p + 1, i);
    std::sort(sl.begin(), sl.end());
    if (sl.size() > 40) return "a part has more than 40 copy bits";
    for (size_t m = 0; m < sl.size(); ++m) {
      mp.slot_bits[p].push_back({std::get<2>(sl[m]), std::get<3>(sl[m])});
      local[p][{std::get<2>(sl[m]), std::get<3>(sl[m])}] = (int)m;
    }
  }
  // gate lists per part
  std::vector<HalfGateLists> hl(mp.t);
  for (auto& H : hl) {
    H.nondiag.assign(c.depth, {});
    H.tmask.assign(c.depth, 0);
    H.cz.assign(c.depth, {});
    H.cuts.assign(c.depth, {});
    H.ucuts.assign(c.depth, {});
  }
  for (const Gate& g : c.gates) {
    const int p = part_of[g.q1];
    const int o = mp.offset[p];
    if (g.code == G_CZ) {
      const int pb = part_of[g.q2];
      if (pb == p) {
        hl[p].cz[g.t].emplace_back(g.q1 - o, g.q2 - o);
      } else {
        const auto jb = where[{g.t, g.q1}];
        hl[p].cuts[g.t].push_back({g.q1 - o, local[p][jb], 0});                    // P_l above the boundary
        hl[pb].cuts[g.t].push_back({g.q2 - mp.offset[pb], local[pb][jb], 4});      // Z^l below it
      }
    } else if (g.code == G_T) {
      hl[p].tmask[g.t] |= 1u << (g.q1 - o);
    } else {
      hl[p].nondiag[g.t].emplace_back(g.q1 - o, g.code);
    }
  }
  mp.part.assign(mp.t, CutPlan());
  for (int p = 0; p < mp.t; ++p) {
    CutPlan& P = mp.part[p];
    P.circ = c;
    P.n_u = mp.nq[p];
    P.n_l = 0;
    P.c = (int)mp.slot_bits[p].size();
    P.fuse_qubits = fuse;
    P.pass_order = pass_order;
    std::vector<int> branch, bits;
    for (int t = 0; t < c.depth; ++t)
      if (!hl[p].cuts[t].empty()) {
        branch.push_back(t);
        bits.push_back((int)hl[p].cuts[t].size());
      }
    build_half(c, hl[p], mp.nq[p], branch, bits, fuse, pass_order == 1, P.sched[0], P.plain[0]);
  }
  return "";
}

}  // namespace sim
