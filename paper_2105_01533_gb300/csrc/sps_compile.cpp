// Gate-batch compiler (host). Splits a gate stream at every two-nonzero gate
// (Sec. 3.1) and turns each maximal run of one-nonzero gates into one op list
// applied per element in a single pass (Sec. 3.2, composition of (f, g) pairs).
// Angles are turned into cos/sin here, once, with the host libm, so the device
// evaluates no transcendental function.
#include <algorithm>
#include <cmath>
#include <cstring>

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

}  // namespace

sps_status compile(const sps_gate* gates, size_t ngates, uint32_t nqubits,
                   uint32_t max_fused_ops, std::vector<Pass>* out, size_t* bad, KnownBits* kb,
                   bool expand) {
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
  Pass* run = nullptr;
  Pass* ex = nullptr;
  for (size_t i = 0; i < ngates; ++i) {
    const sps_gate& g = gates[i];
    if (is_branch(g.op)) {
      run = nullptr;
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
        track(g, k);
        continue;
      }
      ex = nullptr;
      p.kind = PASS_BRANCH;
      out->push_back(std::move(p));
      track(g, k);
      continue;
    }
    ex = nullptr;
    track(g, k);
    const uint32_t slots = g.op == SPS_OP_P ? 1u : (g.op == SPS_OP_RZ ? 2u : 0u);
    if (run == nullptr || run->ops.size() >= max_fused_ops || run->phases.size() >= kMaxFusedPhases ||
        run->fire_slots + slots > kMaxFireSlots) {
      Pass p;
      p.kind = PASS_FUSED;
      p.first_gate = i;
      out->push_back(std::move(p));
      run = &out->back();
    }
    lower_perm_diag(g, run);
  }
  for (Pass& p : *out) {
    if (p.kind == PASS_FUSED) encode_ops(p.ops, &p.words);
    if (p.kind == PASS_EXPAND) build_expand(&p);
  }
  if (kb) *kb = k;
  return SPS_OK;
}

void encode_ops(const std::vector<FOp>& ops, std::vector<OpWord>* words) {
  words->clear();
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
      } else {
        OpWord w[3];
        static_assert(sizeof(w) == sizeof(FOp), "FOp is three words");
        std::memcpy(w, &o, sizeof(FOp));
        words->insert(words->end(), w, w + (f == OPS_FLIP128 ? 2 : 3));
      }
    }
    i = j;
  }
}

// ---- bit-sliced form ------------------------------------------------------------
namespace {

struct CL { double re, im; };

}  // namespace

void build_bitslice(const Pass& p, uint32_t nqubits, BsPass* out) {
  *out = BsPass();
  out->nw = (nqubits + 31) / 32;
  bool cnt = false;
  for (const FOp& o : p.ops) cnt = cnt || o.a0 != 0 || o.a1 != 0;
  out->has_cnt = cnt;
  const uint32_t label_rows = 32 * out->nw;
  uint32_t aux = cnt ? 3u : 0u;
  // factor of every aux bit, for the chunk tables
  std::vector<CL> factor;
  if (cnt) {
    const double r = std::sqrt(0.5);
    factor.push_back(CL{r, r});      // counter bit 0: e^{i pi/4}
    factor.push_back(CL{0, 1});      // counter bit 1: e^{i pi/2}
    factor.push_back(CL{-1, 0});     // counter bit 2: e^{i pi}
  }
  for (const FOp& o : p.ops) {
    SOp so;
    std::memset(&so, 0, sizeof(so));
    std::vector<uint8_t> conds;
    for (int w = 0; w < 2; ++w)
      for (int b = 0; b < 64; ++b)
        if ((o.c[w] >> b) & 1ull) conds.push_back((uint8_t)(64 * w + b));
    so.c[0] = so.c[1] = so.c[2] = SOP_ONES;
    for (size_t k = 0; k < conds.size() && k < 3; ++k) so.c[k] = conds[k];
    if (conds.size() > 3) {
      so.kind |= SOP_LIST;
      so.list_off = (uint16_t)out->list.size();
      so.list_n = (uint16_t)(conds.size() - 3);
      out->list.insert(out->list.end(), conds.begin() + 3, conds.end());
    }
    if (o.t[0] | o.t[1]) {
      so.kind |= SOP_FLIP;
      for (int w = 0; w < 2; ++w)
        for (int b = 0; b < 64; ++b)
          if ((o.t[w] >> b) & 1ull) so.t = (uint8_t)(64 * w + b);
    }
    if (o.sbit != NO_SEL) {
      so.kind |= SOP_SEL;
      so.s = o.sbit;
    }
    if (o.a0 || o.a1) {
      so.kind |= SOP_CNT;
      so.a0 = o.a0;
      so.a1 = o.a1;
    }
    if (o.ph != NO_PH) {
      const PhasePair& pp = p.phases[o.ph];
      so.kind |= SOP_FIRE;
      so.f0 = (uint8_t)(label_rows + aux++);
      factor.push_back(CL{pp.re0, pp.im0});
      if (o.sbit != NO_SEL) {
        so.f1 = (uint8_t)(label_rows + aux++);
        factor.push_back(CL{pp.re1, pp.im1});
      }
    }
    out->ops.push_back(so);
  }
  out->aux_bits = aux;
  out->na = (aux + 31) / 32;
  // unused condition slots read the all-ones row that follows the aux rows
  const uint8_t ones = (uint8_t)(32 * (out->nw + out->na));
  for (SOp& so : out->ops)
    for (int k = 0; k < 3; ++k)
      if (so.c[k] == SOP_ONES) so.c[k] = ones;
  // chunk tables by doubling: entry idx = entry (idx without its top bit) times
  // the factor of that bit, one complex product each
  const uint32_t nch = out->nchunks();
  out->tables.assign((size_t)nch * 256 * 2, 0.0);
  for (uint32_t c = 0; c < nch; ++c) {
    double* t = &out->tables[(size_t)c * 256 * 2];
    t[0] = 1.0;
    for (uint32_t b = 0; b < 8; ++b) {
      const uint32_t bit = 8 * c + b;
      const double fr = bit < aux ? (double)factor[bit].re : 1.0;
      const double fi = bit < aux ? (double)factor[bit].im : 0.0;
      for (uint32_t u = 0; u < (1u << b); ++u) {
        const uint32_t v = u | (1u << b);
        t[2 * v] = t[2 * u] * fr - t[2 * u + 1] * fi;
        t[2 * v + 1] = t[2 * u] * fi + t[2 * u + 1] * fr;
      }
    }
  }
}

}  // namespace sps
