// Gate-batch compiler (host). Splits a gate stream at every two-nonzero gate
// (Sec. 3.1) and turns each maximal run of one-nonzero gates into one op list
// applied per element in a single pass (Sec. 3.2, composition of (f, g) pairs).
// Angles are turned into cos/sin here, once, with the host libm, so the device
// evaluates no transcendental function.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <utility>
#include <vector>

#include "sps_internal.h"

namespace sps {
namespace {

struct Mask128 {
  uint64_t w[2] = {0, 0};
  void set(uint32_t q) { w[q >> 6] |= 1ull << (q & 63); }
  bool has(uint32_t q) const { return (w[q >> 6] >> (q & 63)) & 1ull; }
};

bool in_range(const uint64_t m[2], uint32_t nq) {
  const uint64_t lim0 = nq >= 64 ? ~0ull : ((1ull << nq) - 1);
  const uint64_t lim1 = nq <= 64 ? 0ull : (nq >= 128 ? ~0ull : ((1ull << (nq - 64)) - 1));
  return (m[0] & ~lim0) == 0 && (m[1] & ~lim1) == 0;
}

bool is_branch(uint8_t op) {
  return op == SPS_OP_H || op == SPS_OP_RX || op == SPS_OP_RY || op == SPS_OP_GIVENS;
}

bool check(const sps_gate& g, uint32_t nq) {
  if (g.op < SPS_OP_X || g.op > SPS_OP_GIVENS) return false;
  if (g.reserved0 != 0 || g.reserved1 != 0) return false;
  if (g.t0 >= nq || !in_range(g.cmask, nq)) return false;
  if ((g.cmask[g.t0 >> 6] >> (g.t0 & 63)) & 1ull) return false;
  if (g.op == SPS_OP_GIVENS) {
    if (g.t1 >= nq || g.t1 == g.t0) return false;
    if ((g.cmask[g.t1 >> 6] >> (g.t1 & 63)) & 1ull) return false;
  }
  if (!std::isfinite(g.theta)) return false;
  return true;
}

FOp make_op(const uint64_t cmask[2]) {
  FOp o;
  std::memset(&o, 0, sizeof(o));
  o.c[0] = cmask[0];
  o.c[1] = cmask[1];
  o.sbit = NO_SEL;
  o.ph = NO_PH;
  return o;
}

// Appends the ops of one phase/permutation gate to the pass.
void lower_perm_diag(const sps_gate& g, Pass* p) {
  Mask128 tgt;
  tgt.set(g.t0);
  FOp o = make_op(g.cmask);
  switch (g.op) {
    case SPS_OP_X:   // flip the target
      o.t[0] = tgt.w[0]; o.t[1] = tgt.w[1];
      p->has_perm = true;
      break;
    case SPS_OP_Y:   // |0> -> i|1>, |1> -> -i|0>: phase by the old bit, then flip
      o.t[0] = tgt.w[0]; o.t[1] = tgt.w[1];
      o.sbit = static_cast<uint8_t>(g.t0);
      o.a0 = 2; o.a1 = 6;
      p->has_perm = p->has_phase = true;
      break;
    case SPS_OP_Z: case SPS_OP_S: case SPS_OP_SDG: case SPS_OP_T: case SPS_OP_TDG: {
      // diag(1, e^{i pi a / 4}): condition = controls and the target bit
      o.c[0] |= tgt.w[0]; o.c[1] |= tgt.w[1];
      const uint8_t steps[] = {0, 0, 0, 4, 2, 6, 1, 7};
      o.a0 = steps[g.op];
      p->has_phase = true;
      break;
    }
    case SPS_OP_P: {  // diag(1, e^{i theta})
      o.c[0] |= tgt.w[0]; o.c[1] |= tgt.w[1];
      PhasePair pp{std::cos(g.theta), std::sin(g.theta), 1.0, 0.0};
      o.ph = static_cast<uint16_t>(p->phases.size());
      p->phases.push_back(pp);
      p->has_phase = true;
      p->fire_slots += 1;
      break;
    }
    case SPS_OP_RZ: {  // diag(e^{-i theta/2}, e^{i theta/2}) selected by the target bit
      const double c = std::cos(0.5 * g.theta), s = std::sin(0.5 * g.theta);
      PhasePair pp{c, -s, c, s};
      o.sbit = static_cast<uint8_t>(g.t0);
      o.ph = static_cast<uint16_t>(p->phases.size());
      p->phases.push_back(pp);
      p->has_phase = true;
      p->fire_slots += 2;
      break;
    }
    default:
      break;
  }
  set_fop_kind(o);
  p->ops.push_back(o);
}

void lower_branch(const sps_gate& g, Pass* p) {
  BranchOp& b = p->br;
  std::memset(&b, 0, sizeof(b));
  b.c[0] = g.cmask[0];
  b.c[1] = g.cmask[1];
  Mask128 m;
  m.set(g.t0);
  b.sbit = g.t0;
  if (g.op == SPS_OP_GIVENS) {
    m.set(g.t1);
    b.qbit = g.t1;
    b.givens = 1;
  }
  b.m[0] = m.w[0];
  b.m[1] = m.w[1];
  const double r = std::sqrt(0.5);
  const double c = std::cos(0.5 * g.theta), s = std::sin(0.5 * g.theta);
  double mr[2][2] = {{1, 0}, {0, 1}}, mi[2][2] = {{0, 0}, {0, 0}};
  b.real_m = 1;
  switch (g.op) {
    case SPS_OP_H:
      mr[0][0] = r; mr[0][1] = r; mr[1][0] = r; mr[1][1] = -r;
      break;
    case SPS_OP_RX:   // [[c, -i s], [-i s, c]]
      mr[0][0] = c; mr[1][1] = c; mr[0][1] = 0; mr[1][0] = 0;
      mi[0][1] = -s; mi[1][0] = -s;
      b.real_m = 0;
      break;
    case SPS_OP_RY:   // [[c, -s], [s, c]]
      mr[0][0] = c; mr[0][1] = -s; mr[1][0] = s; mr[1][1] = c;
      break;
    case SPS_OP_GIVENS: {
      const double cg = std::cos(g.theta), sg = std::sin(g.theta);
      mr[0][0] = cg; mr[0][1] = -sg; mr[1][0] = sg; mr[1][1] = cg;
      break;
    }
    default:
      break;
  }
  std::memcpy(b.m_re, mr, sizeof(mr));
  std::memcpy(b.m_im, mi, sizeof(mi));
}

// ---- known-constant qubits ------------------------------------------------------
bool kb_has(const KnownBits& k, uint32_t q) { return (k.known[q >> 6] >> (q & 63)) & 1ull; }
bool kb_val(const KnownBits& k, uint32_t q) { return (k.val[q >> 6] >> (q & 63)) & 1ull; }
void kb_forget(KnownBits& k, uint32_t q) { k.known[q >> 6] &= ~(1ull << (q & 63)); }

// Controls: 1 = all known 1 (the gate acts everywhere), 0 = some known 0 (the
// gate acts nowhere), -1 = depends on the entry.
int controls_state(const sps_gate& g, const KnownBits& k) {
  const uint64_t zero = (g.cmask[0] & k.known[0] & ~k.val[0]) | (g.cmask[1] & k.known[1] & ~k.val[1]);
  if (zero) return 0;
  const uint64_t unknown = (g.cmask[0] & ~k.known[0]) | (g.cmask[1] & ~k.known[1]);
  return unknown ? -1 : 1;
}

// Advances the knowledge over one gate (never claims more than holds: a qubit
// stays known only if the gate cannot change it in any label).
void track(const sps_gate& g, KnownBits& k) {
  const int cs = controls_state(g, k);
  if (cs == 0) return;
  switch (g.op) {
    case SPS_OP_X: case SPS_OP_Y:
      if (cs == 1 && kb_has(k, g.t0)) k.val[g.t0 >> 6] ^= 1ull << (g.t0 & 63);
      else kb_forget(k, g.t0);
      break;
    case SPS_OP_H: case SPS_OP_RX: case SPS_OP_RY:
      kb_forget(k, g.t0);
      break;
    case SPS_OP_GIVENS:
      if (kb_has(k, g.t0) && kb_has(k, g.t1) && kb_val(k, g.t0) == kb_val(k, g.t1)) break;
      kb_forget(k, g.t0);
      kb_forget(k, g.t1);
      break;
    default:   // diagonal gates keep every label
      break;
  }
}

// A branching gate joins an expansion pass if it acts on every entry and only
// flips qubits known constant: then no entry has a partner.
bool expandable(const sps_gate& g, const KnownBits& k) {
  if (controls_state(g, k) != 1 || !kb_has(k, g.t0)) return false;
  if (g.op == SPS_OP_GIVENS)
    return kb_has(k, g.t1) && kb_val(k, g.t0) != kb_val(k, g.t1);
  return true;
}

// Per-chunk tables of an expansion pass: for chunk choices u, the product of
// M_j[x_j ^ u_j][x_j] (the entry taking the amplitude from the selector value
// x_j to the chosen output) over the chunk's gates in order, and the xor of
// the chosen flips. Built by doubling, one complex product per entry; each
// entry carries at most 8 roundings.
void build_expand(Pass* p) {
  p->ex_d = (uint32_t)p->ex_ops.size();
  const uint32_t nch = p->ex_chunks();
  p->ex_f.assign((size_t)nch * 256 * 2, 0.0);
  p->ex_m.assign((size_t)nch * 256 * 2, 0ull);
  p->ex_real = true;
  for (const BranchOp& b : p->ex_ops) p->ex_real = p->ex_real && b.real_m;
  for (uint32_t ch = 0; ch < nch; ++ch) {
    const uint32_t j0 = ch * kExpandChunk;
    const uint32_t g = std::min<uint32_t>(kExpandChunk, p->ex_d - j0);
    double* f = &p->ex_f[(size_t)ch * 256 * 2];
    uint64_t* m = &p->ex_m[(size_t)ch * 256 * 2];
    f[0] = 1.0;
    for (uint32_t b = 0; b < g; ++b) {   // entries [0, 2^b) hold the first b gates
      const BranchOp& op = p->ex_ops[j0 + b];
      const uint32_t x = p->ex_x[j0 + b];
      for (uint32_t u = 0; u < (1u << b); ++u) {
        const double fr = f[2 * u], fi = f[2 * u + 1];
        const uint64_t m0 = m[2 * u], m1 = m[2 * u + 1];
        for (uint32_t cb = 0; cb < 2; ++cb) {   // entry u (cb = 0) and u + 2^b (cb = 1)
          const uint32_t row = x ^ cb, v = u | (cb << b);
          const double er = op.m_re[row][x], ei = op.m_im[row][x];
          f[2 * v] = fr * er - fi * ei;
          f[2 * v + 1] = fr * ei + fi * er;
          m[2 * v] = m0 ^ (cb ? op.m[0] : 0ull);
          m[2 * v + 1] = m1 ^ (cb ? op.m[1] : 0ull);
        }
      }
    }
  }
}

// ---- known qubits in fused runs ---------------------------------------------------
// Appends a pure flip (condition c, targets t) to the run. It merges into the
// previous op when that is a pure flip with the same condition that flips no
// qubit of the condition: the two then act as one flip of both targets.
void append_flip(Pass* run, uint64_t c0, uint64_t c1, uint64_t t0, uint64_t t1) {
  if (!run->ops.empty()) {
    FOp& prev = run->ops.back();
    if ((prev.kind & FOP_FLIP) && (prev.kind & ~(FOP_FLIP | FOP_HI)) == 0 && prev.c[0] == c0 &&
        prev.c[1] == c1 && ((prev.t[0] & c0) | (prev.t[1] & c1)) == 0) {
      prev.t[0] ^= t0;
      prev.t[1] ^= t1;
      set_fop_kind(prev);
      if ((prev.t[0] | prev.t[1]) == 0) run->ops.pop_back();   // the two cancel
      return;
    }
  }
  const uint64_t cm[2] = {c0, c1};
  FOp o = make_op(cm);
  o.t[0] = t0;
  o.t[1] = t1;
  set_fop_kind(o);
  run->ops.push_back(o);
}

// Lowers one phase/permutation gate with the qubits known before it resolved:
// a gate with a control known 0 (or a phase gate whose target is known 0) does
// nothing; known controls (all 1) leave the condition; an unconditional flip of
// a known qubit only toggles its value, recorded in pending and applied to the
// labels later by one flip (the device sees a known qubit's true value only
// where an op reads or conditionally flips it, which materialises it first).
void lower_known(const sps_gate& g, Pass* run, const KnownBits& k, uint64_t pending[2]) {
  if (controls_state(g, k) == 0) return;
  sps_gate h = g;
  h.cmask[0] &= ~k.known[0];
  h.cmask[1] &= ~k.known[1];
  const uint32_t t = g.t0;
  const uint64_t tb0 = t < 64 ? 1ull << t : 0ull, tb1 = t >= 64 ? 1ull << (t - 64) : 0ull;
  auto materialize = [&]() {
    const uint64_t m0 = pending[0] & tb0, m1 = pending[1] & tb1;
    if (m0 | m1) {
      append_flip(run, 0ull, 0ull, m0, m1);
      pending[0] ^= m0;
      pending[1] ^= m1;
    }
  };
  switch (g.op) {
    case SPS_OP_X:
      if ((h.cmask[0] | h.cmask[1]) == 0 && kb_has(k, t)) {
        pending[0] ^= tb0;
        pending[1] ^= tb1;
        return;
      }
      materialize();
      append_flip(run, h.cmask[0], h.cmask[1], tb0, tb1);
      return;
    case SPS_OP_Z: case SPS_OP_S: case SPS_OP_SDG: case SPS_OP_T: case SPS_OP_TDG:
    case SPS_OP_P: {
      if (kb_has(k, t) && !kb_val(k, t)) return;   // the target is 0 everywhere
      lower_perm_diag(h, run);
      if (kb_has(k, t)) {                           // the target is 1 everywhere
        FOp& o = run->ops.back();
        o.c[0] &= ~tb0;
        o.c[1] &= ~tb1;
        set_fop_kind(o);
      }
      return;
    }
    default:   // Y and Rz read the target's value on the device
      materialize();
      lower_perm_diag(h, run);
      return;
  }
}

// ---- gate commuting queues (Sec. 3.3, Fig. 1) ------------------------------------
// Queues per qubit an H, an Rx and an Ry; the pending operation on qubit q is
// Ry(ay) Rx(ax) H^h (H first), above a queue of phase/permutation gates (applied
// before all of them). An incoming gate is commuted down through the queues of
// its qubits with the identities H H = 1, Rx(a) Rx(b) = Rx(a + b), Ry likewise,
// H Ry(t) = Ry(-t) H, X Ry(t) = Ry(-t) X, Z Ry(t) = Ry(-t) Z, Z Rx(t) = Rx(-t) Z,
// X commutes with Rx, and X H = H Z, Z H = H X (with controls where they hold:
// C-X and C-Z through H on the target). Where no such identity applies, the
// qubit's queue is flushed: the phase/permutation queue, then its H, Rx, Ry are
// emitted. At the end everything is flushed, so the stream computes the same
// state; gates that cancel or merge are never run.
class Commuter {
 public:
  Commuter(uint32_t n, std::vector<sps_gate>* out, std::vector<size_t>* origin)
      : q_(n), out_(out), origin_(origin) {}

  void push(const sps_gate& g, size_t idx) {
    const uint32_t t = g.t0;
    const bool controlled = (g.cmask[0] | g.cmask[1]) != 0;
    if (is_branch(g.op)) {
      if (controlled || g.op == SPS_OP_GIVENS) {
        flush_qubit(t);
        if (g.op == SPS_OP_GIVENS) flush_qubit(g.t1);
        flush_controls(g);
        flush_perm();
        emit(g, idx);
        return;
      }
      Queue& e = q_[t];
      if (g.op == SPS_OP_H) {
        if (e.rx) flush_qubit(t);
        if (e.ry) e.ay = -e.ay;
        e.h = !e.h;
        if (e.h) e.oh = idx;
      } else if (g.op == SPS_OP_RX) {
        if (e.ry) flush_qubit(t);
        if (e.rx) {
          e.ax += g.theta;
        } else {
          e.rx = true;
          e.ax = g.theta;
          e.ox = idx;
        }
      } else {   // Ry
        if (e.ry) {
          e.ay += g.theta;
        } else {
          e.ry = true;
          e.ay = g.theta;
          e.oy = idx;
        }
      }
      return;
    }
    flush_controls(g);
    sps_gate h = g;
    Queue& e = q_[t];
    if (e.any()) {
      if (g.op == SPS_OP_X) {
        if (e.ry && controlled) flush_qubit(t);
        if (e.ry) e.ay = -e.ay;
        if (e.h) h.op = SPS_OP_Z;   // C-X H = H C-Z (both on the target)
      } else if (g.op == SPS_OP_Z) {
        if ((e.ry || e.rx) && controlled) flush_qubit(t);
        if (e.ry) e.ay = -e.ay;
        if (e.rx) e.ax = -e.ax;
        if (e.h) h.op = SPS_OP_X;   // C-Z H = H C-X
      } else {
        flush_qubit(t);
      }
    }
    perm_.push_back({h, idx});
  }

  void finish() {
    flush_perm();
    for (uint32_t t = 0; t < q_.size(); ++t) emit_queue(t);
  }

 private:
  struct Queue {
    bool h = false, rx = false, ry = false;
    double ax = 0.0, ay = 0.0;
    size_t oh = 0, ox = 0, oy = 0;
    bool any() const { return h || rx || ry; }
  };

  void emit(const sps_gate& g, size_t idx) {
    out_->push_back(g);
    origin_->push_back(idx);
  }
  void flush_perm() {
    for (const auto& pg : perm_) emit(pg.first, pg.second);
    perm_.clear();
  }
  void emit_queue(uint32_t t) {
    Queue& e = q_[t];
    sps_gate g;
    std::memset(&g, 0, sizeof(g));
    g.t0 = (uint16_t)t;
    if (e.h) {
      g.op = SPS_OP_H;
      emit(g, e.oh);
    }
    if (e.rx) {
      g.op = SPS_OP_RX;
      g.theta = e.ax;
      emit(g, e.ox);
    }
    if (e.ry) {
      g.op = SPS_OP_RY;
      g.theta = e.ay;
      emit(g, e.oy);
    }
    e = Queue();
  }
  void flush_qubit(uint32_t t) {
    if (!q_[t].any()) return;
    flush_perm();
    emit_queue(t);
  }
  void flush_controls(const sps_gate& g) {
    for (int w = 0; w < 2; ++w)
      for (uint64_t m = g.cmask[w]; m; m &= m - 1) flush_qubit(64 * w + (uint32_t)__builtin_ctzll(m));
  }

  std::vector<Queue> q_;
  std::vector<std::pair<sps_gate, size_t>> perm_;
  std::vector<sps_gate>* out_;
  std::vector<size_t>* origin_;
};

}  // namespace

sps_status commute_gates(const sps_gate* gates, size_t ngates, uint32_t nqubits,
                         std::vector<sps_gate>* out, std::vector<size_t>* origin, size_t* bad) {
  out->clear();
  origin->clear();
  for (size_t i = 0; i < ngates; ++i) {
    if (!check(gates[i], nqubits)) {
      if (bad) *bad = i;
      return SPS_ERR_ARG;
    }
  }
  Commuter c(nqubits, out, origin);
  for (size_t i = 0; i < ngates; ++i) c.push(gates[i], i);
  c.finish();
  return SPS_OK;
}

sps_status compile(const sps_gate* gates, size_t ngates, uint32_t nqubits,
                   uint32_t max_fused_ops, std::vector<Pass>* out, size_t* bad, KnownBits* kb,
                   bool expand, bool fold, uint32_t layer_max) {
  if (layer_max > kMaxLayerGates) layer_max = kMaxLayerGates;
  if (max_fused_ops == 0 || max_fused_ops > kMaxFusedOps) max_fused_ops = kDefaultMaxFusedOps;
  out->clear();
  for (size_t i = 0; i < ngates; ++i) {
    if (!check(gates[i], nqubits)) {
      if (bad) *bad = i;
      out->clear();
      return SPS_ERR_ARG;
    }
  }
  KnownBits k = kb ? *kb : KnownBits();
  const bool fold_known = kb != nullptr && fold;
  Pass* run = nullptr;
  Pass* ex = nullptr;
  Pass* lay = nullptr;   // the last pass, while it is a branch or layer pass
  uint64_t pending[2] = {0ull, 0ull};
  auto close_run = [&]() {
    if (run && (pending[0] | pending[1])) append_flip(run, 0ull, 0ull, pending[0], pending[1]);
    pending[0] = pending[1] = 0ull;
    run = nullptr;
  };
  for (size_t i = 0; i < ngates; ++i) {
    const sps_gate& g = gates[i];
    if (is_branch(g.op)) {
      close_run();
      Pass p;
      p.first_gate = i;
      lower_branch(g, &p);
      if (expand && kb && expandable(g, k)) {
        if (ex == nullptr || ex->ex_ops.size() >= kMaxExpandGates) {
          Pass e;
          e.kind = PASS_EXPAND;
          e.first_gate = i;
          out->push_back(std::move(e));
          ex = &out->back();
        }
        ex->ex_ops.push_back(p.br);
        ex->ex_x.push_back(kb_val(k, g.t0) ? 1 : 0);
        lay = nullptr;
        track(g, k);
        continue;
      }
      ex = nullptr;
      Mask128 sup;
      sup.w[0] = g.cmask[0];
      sup.w[1] = g.cmask[1];
      sup.set(g.t0);
      if (g.op == SPS_OP_GIVENS) sup.set(g.t1);
      if (lay != nullptr) {
        const size_t have = lay->kind == PASS_LAYER ? lay->lay.size() : 1;
        if (have < layer_max && ((lay->sup[0] & sup.w[0]) | (lay->sup[1] & sup.w[1])) == 0) {
          if (lay->kind == PASS_BRANCH) {
            lay->kind = PASS_LAYER;
            lay->lay.push_back(lay->br);
            lay->lay_gate.push_back(lay->first_gate);
          }
          lay->lay.push_back(p.br);
          lay->lay_gate.push_back(i);
          lay->sup[0] |= sup.w[0];
          lay->sup[1] |= sup.w[1];
          track(g, k);
          continue;
        }
      }
      p.kind = PASS_BRANCH;
      p.sup[0] = sup.w[0];
      p.sup[1] = sup.w[1];
      out->push_back(std::move(p));
      lay = &out->back();
      track(g, k);
      continue;
    }
    ex = nullptr;
    lay = nullptr;
    const uint32_t slots = g.op == SPS_OP_P ? 1u : (g.op == SPS_OP_RZ ? 2u : 0u);
    // folding may add two flips (a materialised known qubit, the pending ones)
    const size_t room = fold_known ? 2 : 0;
    if (run == nullptr || run->ops.size() + room >= max_fused_ops ||
        run->phases.size() >= kMaxFusedPhases || run->fire_slots + slots > kMaxFireSlots) {
      close_run();
      Pass p;
      p.kind = PASS_FUSED;
      p.first_gate = i;
      out->push_back(std::move(p));
      run = &out->back();
    }
    if (fold_known)
      lower_known(g, run, k, pending);
    else
      lower_perm_diag(g, run);
    ++run->ngates;
    track(g, k);
  }
  close_run();
  for (Pass& p : *out) {
    if (p.kind == PASS_FUSED) encode_ops(&p);
    if (p.kind == PASS_EXPAND) build_expand(&p);
  }
  if (kb) *kb = k;
  return SPS_OK;
}

void encode_ops(Pass* p) {
  const std::vector<FOp>& ops = p->ops;
  std::vector<OpWord>* words = &p->words;
  words->clear();
  p->has_perm = p->has_phase = false;
  for (const FOp& o : ops) {
    p->has_perm = p->has_perm || (o.kind & FOP_FLIP);
    p->has_phase = p->has_phase || (o.kind & (FOP_CNT | FOP_PH));
  }
  // fire slots in op order; slot k's factor is the phase its op applies
  std::vector<double> factor;
  auto form = [](const FOp& o) {
    if (o.kind == FOP_FLIP) return OPS_FLIP64;
    if (o.kind == (FOP_FLIP | FOP_HI)) return OPS_FLIP128;
    return OPS_GEN;
  };
  size_t i = 0;
  while (i < ops.size()) {
    const uint32_t f = form(ops[i]);
    size_t j = i;
    while (j < ops.size() && form(ops[j]) == f) ++j;
    words->push_back(OpWord{f, (uint32_t)(j - i), 0u, 0u});
    for (size_t k = i; k < j; ++k) {
      const FOp& o = ops[k];
      if (f == OPS_FLIP64) {
        words->push_back(OpWord{(uint32_t)o.c[0], (uint32_t)(o.c[0] >> 32), (uint32_t)o.t[0],
                                (uint32_t)(o.t[0] >> 32)});
        continue;
      }
      FOp e = o;
      if (f == OPS_GEN) {
        uint32_t f0 = 0xFF, f1 = 0xFF;
        if (o.ph != NO_PH) {
          const PhasePair& pp = p->phases[o.ph];
          f0 = (uint32_t)(factor.size() / 2);
          factor.push_back(pp.re0);
          factor.push_back(pp.im0);
          if (o.sbit != NO_SEL) {
            f1 = (uint32_t)(factor.size() / 2);
            factor.push_back(pp.re1);
            factor.push_back(pp.im1);
          }
        }
        e.ph = (uint16_t)(f0 | (f1 << 8));
      }
      OpWord w[3];
      static_assert(sizeof(w) == sizeof(FOp), "FOp is three words");
      std::memcpy(w, &e, sizeof(FOp));
      words->insert(words->end(), w, w + (f == OPS_FLIP128 ? 2 : 3));
    }
    i = j;
  }
  // per-8-slot tables by doubling: entry v = entry (v without its top bit)
  // times the factor of that bit
  const uint32_t nslots = (uint32_t)(factor.size() / 2);
  const uint32_t nch = (nslots + 7) / 8;
  p->ftab.assign((size_t)nch * 256 * 2, 0.0);
  for (uint32_t c = 0; c < nch; ++c) {
    double* t = &p->ftab[(size_t)c * 256 * 2];
    t[0] = 1.0;
    for (uint32_t b = 0; b < 8; ++b) {
      const uint32_t slot = 8 * c + b;
      const double fr = slot < nslots ? factor[2 * slot] : 1.0;
      const double fi = slot < nslots ? factor[2 * slot + 1] : 0.0;
      for (uint32_t u = 0; u < (1u << b); ++u) {
        const uint32_t v = u | (1u << b);
        t[2 * v] = t[2 * u] * fr - t[2 * u + 1] * fi;
        t[2 * v + 1] = t[2 * u] * fi + t[2 * u + 1] * fr;
      }
    }
  }
}

// ---- bit-sliced form ------------------------------------------------------------
namespace {

struct CL { double re, im; };

// x in [-1, 1] as fixed point with 2^62 = 1 (exact: a double has 53 bits)
long long to_q62(double x) { return std::llround(std::ldexp(x, 62)); }

}  // namespace

namespace {
void build_bitslice_rows(const Pass& p, uint32_t nqubits, const uint64_t extra[2], bool all_out,
                         BsPass* out);
}  // namespace

void build_bitslice(const Pass& p, uint32_t nqubits, BsPass* out) {
  const uint64_t none[2] = {0ull, 0ull};
  build_bitslice_rows(p, nqubits, none, false, out);
}

bool build_bitslice_expand(const Pass& ex, const Pass& run, uint32_t nqubits, double eps,
                           BsPass* out) {
  if (ex.kind != PASS_EXPAND || run.kind != PASS_FUSED || ex.ex_d == 0 || ex.ex_d > kMaxExpandGates)
    return false;
  Pass comb;
  comb.kind = PASS_FUSED;
  comb.first_gate = ex.first_gate;
  comb.ngates = run.ngates;
  comb.has_perm = true;
  comb.has_phase = run.has_phase;
  uint64_t targets[2] = {0ull, 0ull};
  double cr = 1.0, ci = 0.0, least = 1.0;
  std::vector<int> choice_qubit(ex.ex_d);
  for (uint32_t j = 0; j < ex.ex_d; ++j) {
    const BranchOp& op = ex.ex_ops[j];
    if (__builtin_popcountll(op.m[0]) + __builtin_popcountll(op.m[1]) != 1) return false;
    if (ex.ex_x[j] != 0) return false;   // from |0...0>: every selector starts at 0
    const uint32_t q = op.m[0] ? (uint32_t)__builtin_ctzll(op.m[0]) : 64u + (uint32_t)__builtin_ctzll(op.m[1]);
    if ((targets[q >> 6] >> (q & 63u)) & 1ull) return false;
    targets[q >> 6] |= 1ull << (q & 63u);
    choice_qubit[j] = (int)q;
    // output bit b (= choice bit j) takes the factor M[b][0]
    const double r0 = op.m_re[0][0], i0 = op.m_im[0][0], r1 = op.m_re[1][0], i1 = op.m_im[1][0];
    const double a0 = std::hypot(r0, i0), a1 = std::hypot(r1, i1);
    least *= std::min(a0, a1);
    if (r0 == r1 && i0 == i1) {   // the same factor either way: into the common factor
      const double nr = cr * r0 - ci * i0, ni = cr * i0 + ci * r0;
      cr = nr;
      ci = ni;
    } else {   // a phase slot on the qubit: M[0][0] where it is 0, M[1][0] where it is 1
      FOp o;
      std::memset(&o, 0, sizeof(o));
      o.sbit = (uint8_t)q;
      o.ph = (uint16_t)comb.phases.size();
      set_fop_kind(o);
      comb.ops.push_back(o);
      comb.phases.push_back(PhasePair{r0, i0, r1, i1});
      comb.has_phase = true;
    }
  }
  if (!(least > 2.0 * eps) || least == 0.0) return false;
  // the run's ops after the prefix, their phase pairs after the prefix's
  const size_t base = comb.phases.size();
  for (const FOp& o : run.ops) {
    FOp c = o;
    if (c.ph != NO_PH) c.ph = (uint16_t)(c.ph + base);
    comb.ops.push_back(c);
  }
  comb.phases.insert(comb.phases.end(), run.phases.begin(), run.phases.end());
  if (comb.phases.size() > kMaxFusedPhases + kMaxExpandGates) return false;
  build_bitslice_rows(comb, nqubits, targets, true, out);
  if (out->aux_bits > kBsDirectBits) return false;   // the phase from one table
  out->expand = true;
  out->ex_d = ex.ex_d;
  out->c_re = cr;
  out->c_im = ci;
  out->row_choice.assign(out->nrows, (int8_t)-1);
  for (uint32_t j = 0; j < ex.ex_d; ++j) {
    const int q = choice_qubit[j];
    const uint8_t r = out->row_of[q >> 5][q & 31];
    if (r == kNoRow) return false;
    out->row_choice[r] = (int8_t)j;
  }
  return out->aux_bits <= kMaxAuxBits && out->op_words() <= kBsMaxOps;
}

namespace {

void build_bitslice_rows(const Pass& p, uint32_t nqubits, const uint64_t extra[2], bool all_out,
                         BsPass* out) {
  *out = BsPass();
  BsPass& b = *out;
  b.ops.reserve(p.ops.size() + p.ops.size() / 4 + 8);
  b.nw = (nqubits + 31) / 32;
  std::memset(b.row_of, kNoRow, sizeof(b.row_of));
  // qubits the ops read (conditions, selectors) and flip
  uint64_t used[2] = {extra[0], extra[1]}, flipped[2] = {0ull, 0ull};
  bool cnt = false;
  for (const FOp& o : p.ops) {
    for (int w = 0; w < 2; ++w) {
      used[w] |= o.c[w] | o.t[w];
      flipped[w] |= o.t[w];
    }
    if (o.sbit != NO_SEL) used[o.sbit >> 6] |= 1ull << (o.sbit & 63u);
    cnt = cnt || o.a0 != 0 || o.a1 != 0;
  }
  // a 64-bit half with a flipped bit is written back whole: every valid bit of
  // it gets a row (its other bits are 0 in every label). With all_out every
  // half is written, and only the used bits have rows (the others are 0)
  for (int h = 0; h < 2; ++h) {
    if (all_out) {
      for (int k = 0; k < 2; ++k)
        if (32u * (2 * h + k) < nqubits) b.word_out |= 1u << (2 * h + k);
      continue;
    }
    if (!flipped[h]) continue;
    const uint64_t valid = nqubits >= 64 * (h + 1) ? ~0ull
                         : (nqubits <= 64u * h ? 0ull : ((1ull << (nqubits - 64 * h)) - 1));
    used[h] |= valid;
    for (int k = 0; k < 2; ++k)
      if ((valid >> (32 * k)) & 0xFFFFFFFFull) b.word_out |= 1u << (2 * h + k);
  }
  uint32_t row = 0;
  for (uint32_t w = 0; w < 4; ++w) {
    const uint32_t bits = (uint32_t)(used[w >> 1] >> (32 * (w & 1u)));
    b.word_bits[w] = bits;
    for (uint32_t j = 0; j < 32; ++j)
      if ((bits >> j) & 1u) b.row_of[w][j] = (uint8_t)row++;
  }
  b.label_rows = row;
  auto row_q = [&](uint32_t q) { return b.row_of[q >> 5][q & 31u]; };
  b.has_cnt = cnt;
  b.aux_row0 = row;
  uint32_t aux = cnt ? 3u : 0u;
  std::vector<CL> factor;
  if (cnt) {
    const double r = std::sqrt(0.5);
    factor.push_back(CL{r, r});      // counter bit 0: e^{i pi/4}
    factor.push_back(CL{0, 1});      // counter bit 1: e^{i pi/2}
    factor.push_back(CL{-1, 0});     // counter bit 2: e^{i pi}
  }
  for (const FOp& o : p.ops)
    if (o.ph != NO_PH) aux += o.sbit != NO_SEL ? 2u : 1u;
  b.aux_bits = aux;
  const uint8_t scratch = (uint8_t)(b.aux_row0 + aux);
  b.ones_row = scratch + 1u;
  b.nrows = b.ones_row + 1u;
  uint32_t next_aux = b.aux_row0 + (cnt ? 3u : 0u);
  const uint8_t ones = (uint8_t)b.ones_row;
  for (const FOp& o : p.ops) {
    SOp so;
    std::memset(&so, 0, sizeof(so));
    so.c[0] = so.c[1] = so.c[2] = ones;
    so.t = so.s = so.f0 = so.f1 = kNoRow;
    uint8_t conds[130];   // at most 128 condition qubits, then the scratch row
    size_t nconds = 0;
    for (uint32_t w = 0; w < 2; ++w)
      for (uint64_t m = o.c[w]; m; m &= m - 1)
        conds[nconds++] = row_q(64 * w + (uint32_t)__builtin_ctzll(m));
    if (nconds > 3) {
      // AND the conditions past the second into the scratch row, three at a time
      size_t k = 2;
      bool first = true;
      while (k < nconds) {
        SOp a;
        std::memset(&a, 0, sizeof(a));
        a.kind = SOP_AND;
        a.t = scratch;
        a.s = a.f0 = a.f1 = kNoRow;
        a.c[0] = first ? conds[k++] : scratch;
        a.c[1] = k < nconds ? conds[k++] : ones;
        a.c[2] = k < nconds ? conds[k++] : ones;
        first = false;
        b.ops.push_back(a);
      }
      nconds = 3;
      conds[2] = scratch;
    }
    for (size_t k = 0; k < nconds; ++k) so.c[k] = conds[k];
    uint8_t tbits[128];   // a merged flip has several targets, one condition
    size_t ntbits = 0;
    for (uint32_t w = 0; w < 2; ++w)
      for (uint64_t m = o.t[w]; m; m &= m - 1)
        tbits[ntbits++] = row_q(64 * w + (uint32_t)__builtin_ctzll(m));
    if (ntbits > 0) {
      so.kind |= SOP_FLIP;
      so.t = tbits[0];
    }
    if (o.sbit != NO_SEL) {
      so.kind |= SOP_SEL;
      so.s = row_q(o.sbit);
    }
    if (o.a0 || o.a1) {
      so.kind |= SOP_CNT;
      so.a0 = o.a0 & 7u;
      so.a1 = o.a1 & 7u;
    }
    if (o.ph != NO_PH) {
      const PhasePair& pp = p.phases[o.ph];
      so.kind |= SOP_FIRE;
      so.f0 = (uint8_t)next_aux++;
      factor.push_back(CL{pp.re0, pp.im0});
      if (o.sbit != NO_SEL) {
        so.f1 = (uint8_t)next_aux++;
        factor.push_back(CL{pp.re1, pp.im1});
      }
    }
    b.ops.push_back(so);
    // further targets: the same condition (no target is in it), flip only
    for (size_t k = 1; k < ntbits; ++k) {
      SOp x = so;
      x.kind = SOP_FLIP;
      x.t = tbits[k];
      b.ops.push_back(x);
    }
  }
  b.factors.resize(2 * (size_t)aux);
  for (uint32_t i = 0; i < aux; ++i) {
    b.factors[2 * i] = to_q62(factor[i].re);
    b.factors[2 * i + 1] = to_q62(factor[i].im);
  }
  // phase tables: the aux bits in as few chunks of at most kBsMaxChunkBits as
  // possible, split evenly (one table product per extra chunk and entry); up
  // to kBsDirectBits aux bits, two chunks that build one direct table
  if (aux > 0) {
    b.direct = aux <= kBsDirectBits;
    b.nchunks = b.direct ? (aux > 1 ? 2u : 1u) : (aux + kBsMaxChunkBits - 1) / kBsMaxChunkBits;
    uint32_t at = 0;
    for (uint32_t c = 0; c < b.nchunks; ++c) {
      const uint32_t bits = aux / b.nchunks + (c < aux % b.nchunks ? 1u : 0u);
      b.chunk_shift[c] = at;
      b.chunk_bits[c] = bits;
      at += bits;
    }
  }
}

}  // namespace

// The most nonzeros a state can reach from |0...0> through these passes: every
// branching gate at most doubles the count (an expansion of d gates, d
// doublings; a layer, one per gate), never above the capacity.
uint64_t projected_peak(const std::vector<Pass>& passes, uint64_t capacity) {
  uint64_t b = 1, peak = 1;
  for (const Pass& p : passes) {
    uint32_t doublings = 0;
    if (p.kind == PASS_BRANCH) doublings = 1;
    if (p.kind == PASS_EXPAND) doublings = p.ex_d;
    if (p.kind == PASS_LAYER) doublings = (uint32_t)p.lay.size();
    for (uint32_t k = 0; k < doublings && b < capacity; ++k) b *= 2;
    if (b > capacity) b = capacity;
    if (b > peak) peak = b;
    if (peak == capacity) break;
  }
  return peak < capacity ? peak : capacity;
}

}  // namespace sps
