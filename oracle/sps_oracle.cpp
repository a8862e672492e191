// Oracle for the sparse-state gate-application path. TEST INFRASTRUCTURE ONLY:
// it is loaded by the test-suite, by the smoke check and by the CPU-baseline leg
// of the benchmark, never by the product path. It shares no code, header,
// table or constant with the CUDA library; it parses the 32-byte gate record
// with its own definition below.
//
// What it computes (all citations are to arXiv 2105.01533):
//   * Sec. 3: a state sum_b alpha_b |b> is stored as unordered (label, amplitude)
//     pairs, only for alpha_b != 0. Here: std::unordered_map<Key, Cplx>.
//   * Sec. 2.1: |i> = |i_{n-1}> (x) ... (x) |i_0>, so qubit k is bit k of the label.
//   * Sec. 2.1: gate matrices H, S, X, Y, Z, R_P(theta) = exp(-i theta P / 2),
//     and the controlled-gate definition CU = |0><0| (x) 1 + |1><1| (x) U, iterated
//     for several controls.
//   * Sec. 3.1, Eq. 2: a gate with two nonzeros per row acts on the pair (b, b')
//     by a 2x2 matrix; a gate with one nonzero per row maps alpha_b|b> to
//     f(b) alpha_b |g(b)> (Sec. 3.2).
//   * Sec. 3.1: every operation iterates over the old map and inserts into a NEW
//     map (out of place). Two modes:
//       mode 0 (scatter): every old entry adds its contribution(s) into the new
//               map; a label with two contributions receives both.
//       mode 1 (gather, the insert-once rule of Sec. 3.1): every old entry looks
//               up its partner in the old map; if both partners are present only
//               the one whose selector bit is 1 writes the pair.
//     Both give the same result bit for bit (0 + x = x and x + y = y + x in IEEE).
//   * Pruning is not in the paper (it stores alpha != 0 only). After every
//     branching gate an entry is dropped when it is exactly zero or when
//     re*re + im*im < eps*eps (strict). Phase/permutation gates never prune.
//   * Givens(theta) on qubits (p, q) is not in the paper. It acts on the span of
//     {bit p = 0, bit q = 1} (first basis vector) and {bit p = 1, bit q = 0}
//     (second) by [[cos t, -sin t], [sin t, cos t]]; keys with bit p == bit q
//     are unchanged.
//
// No fusion, no reordering, no commuting: one gate at a time, in order.
// Built with -ffp-contract=off so that every product and sum is rounded once.
//
// Also here, as independent checkers for the pins:
//   * a dense 2^n Schroedinger statevector simulator (Sec. 2.2), n <= 26;
//   * a classical evaluator for permutation-only circuits: a key is pushed
//     through X/CNOT/Toffoli/MCX gates one at a time;
//   * a dense simulator restricted to one Hamming-weight sector (every label
//     with k bits set, ranked by the combinatorial number system) for
//     number-conserving circuits (Givens and diagonal gates), n <= 64.

#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <unordered_map>
#include <vector>

namespace {

// ---- gate record, 32 bytes, little-endian -----------------------------------
struct GateRec {
  uint8_t op;
  uint8_t reserved0;
  uint16_t t0;
  uint16_t t1;
  uint16_t reserved1;
  uint64_t cmask[2];  // controls: word 0 = qubits 0..63, word 1 = qubits 64..127
  double theta;
};
static_assert(sizeof(GateRec) == 32, "gate record must be 32 bytes");

enum Op : uint8_t {
  OP_X = 1, OP_Y = 2, OP_Z = 3, OP_S = 4, OP_SDG = 5, OP_T = 6, OP_TDG = 7,
  OP_P = 8, OP_RZ = 9, OP_H = 10, OP_RX = 11, OP_RY = 12, OP_GIVENS = 13,
};

struct Key {
  uint64_t lo, hi;
  bool operator==(const Key& o) const { return lo == o.lo && hi == o.hi; }
};
struct KeyHash {
  size_t operator()(const Key& k) const {
    return std::hash<uint64_t>()(k.lo) ^ (std::hash<uint64_t>()(k.hi) * 0x9E3779B97F4A7C15ull);
  }
};

struct Cplx { double re, im; };

inline Cplx cmul(Cplx a, Cplx b) {
  return Cplx{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
inline Cplx cadd(Cplx a, Cplx b) { return Cplx{a.re + b.re, a.im + b.im}; }

using Map = std::unordered_map<Key, Cplx, KeyHash>;

inline bool bit(const Key& k, unsigned q) {
  return q < 64 ? ((k.lo >> q) & 1u) : ((k.hi >> (q - 64)) & 1u);
}
inline Key flip(Key k, unsigned q) {
  if (q < 64) k.lo ^= (1ull << q); else k.hi ^= (1ull << (q - 64));
  return k;
}
inline bool controls_hold(const Key& k, const GateRec& g) {
  return (k.lo & g.cmask[0]) == g.cmask[0] && (k.hi & g.cmask[1]) == g.cmask[1];
}

struct State {
  unsigned nqubits;
  Map map;
};

enum Kind { PERM_DIAG, BRANCH, INVALID };

Kind kind_of(uint8_t op) {
  switch (op) {
    case OP_X: case OP_Y: case OP_Z: case OP_S: case OP_SDG: case OP_T:
    case OP_TDG: case OP_P: case OP_RZ:
      return PERM_DIAG;
    case OP_H: case OP_RX: case OP_RY: case OP_GIVENS:
      return BRANCH;
    default:
      return INVALID;
  }
}

bool valid(const GateRec& g, unsigned n) {
  if (kind_of(g.op) == INVALID) return false;
  if (g.t0 >= n) return false;
  uint64_t lim[2];
  lim[0] = n >= 64 ? ~0ull : ((1ull << n) - 1);
  lim[1] = n <= 64 ? 0ull : (n >= 128 ? ~0ull : ((1ull << (n - 64)) - 1));
  if ((g.cmask[0] & ~lim[0]) || (g.cmask[1] & ~lim[1])) return false;
  Key t{0, 0};
  t = flip(t, g.t0);
  if ((t.lo & g.cmask[0]) || (t.hi & g.cmask[1])) return false;
  if (g.op == OP_GIVENS) {
    if (g.t1 >= n || g.t1 == g.t0) return false;
    Key u{0, 0};
    u = flip(u, g.t1);
    if ((u.lo & g.cmask[0]) || (u.hi & g.cmask[1])) return false;
  }
  return true;
}

// One-nonzero-per-row gates (Sec. 3.2): alpha_b|b> -> f(b) alpha_b |g(b)>.
// Returns the factor f(b) and writes g(b) to *out_key. Gates are taken one by
// one straight from their matrices (Sec. 2.1).
Cplx perm_diag_action(const GateRec& g, const Key& k, Key* out_key) {
  const double r = std::sqrt(0.5);
  *out_key = k;
  if (!controls_hold(k, g)) return Cplx{1.0, 0.0};
  const bool b = bit(k, g.t0);
  switch (g.op) {
    case OP_X:  // X = [[0,1],[1,0]]
      *out_key = flip(k, g.t0);
      return Cplx{1.0, 0.0};
    case OP_Y:  // Y = [[0,-i],[i,0]]: |0> -> i|1>, |1> -> -i|0>
      *out_key = flip(k, g.t0);
      return b ? Cplx{0.0, -1.0} : Cplx{0.0, 1.0};
    case OP_Z:  // diag(1, -1)
      return b ? Cplx{-1.0, 0.0} : Cplx{1.0, 0.0};
    case OP_S:  // diag(1, i)
      return b ? Cplx{0.0, 1.0} : Cplx{1.0, 0.0};
    case OP_SDG:  // diag(1, -i)
      return b ? Cplx{0.0, -1.0} : Cplx{1.0, 0.0};
    case OP_T:  // diag(1, e^{i pi/4})
      return b ? Cplx{r, r} : Cplx{1.0, 0.0};
    case OP_TDG:  // diag(1, e^{-i pi/4})
      return b ? Cplx{r, -r} : Cplx{1.0, 0.0};
    case OP_P:  // diag(1, e^{i theta}); with one control this is CP(theta)
      return b ? Cplx{std::cos(g.theta), std::sin(g.theta)} : Cplx{1.0, 0.0};
    case OP_RZ: {  // exp(-i theta Z / 2) = diag(e^{-i theta/2}, e^{i theta/2})
      const double c = std::cos(0.5 * g.theta), s = std::sin(0.5 * g.theta);
      return b ? Cplx{c, s} : Cplx{c, -s};
    }
    default:
      return Cplx{1.0, 0.0};
  }
}

// Two-nonzero gates (Sec. 3.1, Eq. 2). For label k with the gate active, the
// pair is (k0, k1) with k0 the label whose selector bit is 0 (for Givens: the
// label with bit p = 0, bit q = 1). M is the 2x2 matrix on (k0, k1).
struct Pair { Key k0, k1; bool sel; };

void branch_matrix(const GateRec& g, Cplx M[2][2]) {
  const double r = std::sqrt(0.5);
  const double c = std::cos(0.5 * g.theta), s = std::sin(0.5 * g.theta);
  switch (g.op) {
    case OP_H:  // sqrt(0.5) [[1,1],[1,-1]]
      M[0][0] = {r, 0}; M[0][1] = {r, 0}; M[1][0] = {r, 0}; M[1][1] = {-r, 0};
      break;
    case OP_RX:  // exp(-i theta X / 2) = [[c, -i s], [-i s, c]]
      M[0][0] = {c, 0}; M[0][1] = {0, -s}; M[1][0] = {0, -s}; M[1][1] = {c, 0};
      break;
    case OP_RY:  // exp(-i theta Y / 2) = [[c, -s], [s, c]]
      M[0][0] = {c, 0}; M[0][1] = {-s, 0}; M[1][0] = {s, 0}; M[1][1] = {c, 0};
      break;
    case OP_GIVENS: {  // [[cos t, -sin t], [sin t, cos t]] on (p=0,q=1), (p=1,q=0)
      const double cg = std::cos(g.theta), sg = std::sin(g.theta);
      M[0][0] = {cg, 0}; M[0][1] = {-sg, 0}; M[1][0] = {sg, 0}; M[1][1] = {cg, 0};
      break;
    }
    default:
      M[0][0] = {1, 0}; M[0][1] = {0, 0}; M[1][0] = {0, 0}; M[1][1] = {1, 0};
  }
}

// Is the 2x2 block active on label k, and if so which pair does k belong to?
bool branch_pair(const GateRec& g, const Key& k, Pair* pr) {
  if (!controls_hold(k, g)) return false;
  if (g.op == OP_GIVENS) {
    const bool bp = bit(k, g.t0), bq = bit(k, g.t1);
    if (bp == bq) return false;  // |00> and |11> are left alone
    const Key other = flip(flip(k, g.t0), g.t1);
    pr->sel = bp;
    pr->k0 = bp ? other : k;
    pr->k1 = bp ? k : other;
    return true;
  }
  const bool b = bit(k, g.t0);
  const Key other = flip(k, g.t0);
  pr->sel = b;
  pr->k0 = b ? other : k;
  pr->k1 = b ? k : other;
  return true;
}

void add_to(Map& m, const Key& k, Cplx v) {
  auto it = m.find(k);
  if (it == m.end()) {
    m.emplace(k, cadd(Cplx{0.0, 0.0}, v));
  } else {
    it->second = cadd(it->second, v);
  }
}

void prune(Map& m, double eps) {
  const double e2 = eps * eps;
  for (auto it = m.begin(); it != m.end();) {
    const double re = it->second.re, im = it->second.im;
    const double mag2 = re * re + im * im;
    if ((re == 0.0 && im == 0.0) || mag2 < e2) it = m.erase(it); else ++it;
  }
}

void apply_perm_diag(State& st, const GateRec& g) {
  Map out;
  out.reserve(st.map.size());
  for (const auto& kv : st.map) {
    Key nk;
    const Cplx f = perm_diag_action(g, kv.first, &nk);
    out.emplace(nk, cmul(f, kv.second));
  }
  st.map.swap(out);
}

// mode 0: scatter form.
void apply_branch_scatter(State& st, const GateRec& g, double eps) {
  Cplx M[2][2];
  branch_matrix(g, M);
  Map out;
  out.reserve(st.map.size() * 2);
  for (const auto& kv : st.map) {
    Pair pr;
    if (!branch_pair(g, kv.first, &pr)) {
      add_to(out, kv.first, kv.second);
      continue;
    }
    const int x = pr.sel ? 1 : 0;
    add_to(out, pr.k0, cmul(M[0][x], kv.second));
    add_to(out, pr.k1, cmul(M[1][x], kv.second));
  }
  prune(out, eps);
  st.map.swap(out);
}

// mode 1: the insert-once gather rule of Sec. 3.1.
void apply_branch_gather(State& st, const GateRec& g, double eps) {
  Cplx M[2][2];
  branch_matrix(g, M);
  Map out;
  out.reserve(st.map.size() * 2);
  for (const auto& kv : st.map) {
    Pair pr;
    if (!branch_pair(g, kv.first, &pr)) {
      out.emplace(kv.first, kv.second);
      continue;
    }
    const Key partner = pr.sel ? pr.k0 : pr.k1;
    auto it = st.map.find(partner);
    if (it != st.map.end() && !pr.sel) continue;  // partner with bit 1 writes the pair
    const Cplx zero{0.0, 0.0};
    const Cplx a0 = pr.sel ? (it != st.map.end() ? it->second : zero) : kv.second;
    const Cplx a1 = pr.sel ? kv.second : (it != st.map.end() ? it->second : zero);
    const Cplx n0 = cadd(cmul(M[0][0], a0), cmul(M[0][1], a1));
    const Cplx n1 = cadd(cmul(M[1][0], a0), cmul(M[1][1], a1));
    out.emplace(pr.k0, n0);
    out.emplace(pr.k1, n1);
  }
  prune(out, eps);
  st.map.swap(out);
}

}  // namespace

extern "C" {

// Status codes of this file: 0 ok, 1 bad argument, 2 buffer too small.

void* orc_create(uint32_t nqubits) {
  if (nqubits < 1 || nqubits > 127) return nullptr;
  State* st = new State;
  st->nqubits = nqubits;
  st->map.emplace(Key{0, 0}, Cplx{1.0, 0.0});
  return st;
}

void orc_destroy(void* h) { delete static_cast<State*>(h); }

void* orc_clone(void* h) {
  State* src = static_cast<State*>(h);
  State* st = new State;
  st->nqubits = src->nqubits;
  st->map = src->map;
  return st;
}

uint32_t orc_nqubits(void* h) { return static_cast<State*>(h)->nqubits; }

uint64_t orc_nnz(void* h) { return static_cast<State*>(h)->map.size(); }

// Applies ngates records in order. Returns 0, or 1 with *bad = index of the
// first invalid record (nothing after it is applied; gates before it are).
// Applies the gates in order. If `updates` is not null it receives the sum over
// gates of the number of stored entries before each gate (the work count the
// benchmark reports as nonzero-amplitude updates).
int orc_apply_counted(void* h, const void* gates, uint64_t ngates, double eps, int mode,
                      uint64_t* bad, uint64_t* updates) {
  State* st = static_cast<State*>(h);
  const GateRec* g = static_cast<const GateRec*>(gates);
  for (uint64_t i = 0; i < ngates; ++i) {
    if (!valid(g[i], st->nqubits)) {
      if (bad) *bad = i;
      return 1;
    }
    if (updates) *updates += st->map.size();
    if (kind_of(g[i].op) == PERM_DIAG) {
      apply_perm_diag(*st, g[i]);
    } else if (mode == 1) {
      apply_branch_gather(*st, g[i], eps);
    } else {
      apply_branch_scatter(*st, g[i], eps);
    }
  }
  return 0;
}

int orc_apply(void* h, const void* gates, uint64_t ngates, double eps, int mode, uint64_t* bad) {
  return orc_apply_counted(h, gates, ngates, eps, mode, bad, nullptr);
}

// Copies the entries out in the map's (unspecified) order.
int orc_get(void* h, uint64_t* hi, uint64_t* lo, double* re, double* im, uint64_t cap) {
  State* st = static_cast<State*>(h);
  if (cap < st->map.size()) return 2;
  uint64_t i = 0;
  for (const auto& kv : st->map) {
    hi[i] = kv.first.hi;
    lo[i] = kv.first.lo;
    re[i] = kv.second.re;
    im[i] = kv.second.im;
    ++i;
  }
  return 0;
}

// Replaces the state by the given entries (later duplicates overwrite earlier).
int orc_set(void* h, const uint64_t* hi, const uint64_t* lo, const double* re,
            const double* im, uint64_t n) {
  State* st = static_cast<State*>(h);
  Map m;
  m.reserve(n);
  for (uint64_t i = 0; i < n; ++i) m[Key{lo[i], hi[i]}] = Cplx{re[i], im[i]};
  st->map.swap(m);
  return 0;
}

// Sum of |alpha_k|^2 over labels with (k & mask) == value.
double orc_probability(void* h, const uint64_t* mask, const uint64_t* value) {
  State* st = static_cast<State*>(h);
  double p = 0.0;
  for (const auto& kv : st->map) {
    if ((kv.first.lo & mask[0]) == value[0] && (kv.first.hi & mask[1]) == value[1])
      p += kv.second.re * kv.second.re + kv.second.im * kv.second.im;
  }
  return p;
}

// Pauli exponential exp(-i theta/2 P) (Sec. 3 lists Pauli exponentials among the
// operations; Sec. 2.1 defines X, Y, Z and R_P(theta) = exp(-i theta P / 2)).
// P is a tensor product of one Pauli per qubit, given by two masks: x (the
// qubit's factor is X or Y) and z (Z or Y); Y = i X Z. On a basis label j,
// X|b> = |1-b>, Z|b> = (-1)^b |b>, Y|b> = i (-1)^b |1-b>, so
//   P|j> = i^nY (-1)^popcount(j & z) |j ^ x>,   nY = popcount(x & z),
// and since P^2 = 1, exp(-i t/2 P)|j> = cos(t/2)|j> - i sin(t/2) P|j>. With
// controls c (disjoint from the string) labels without every control bit set
// are unchanged. Applied out of place into a new map (contributions added),
// then pruned as a branching gate. Returns 1 on bad masks.
int orc_pauli_exp(void* h, const uint64_t* x, const uint64_t* z, const uint64_t* c,
                  double theta, double eps) {
  State* st = static_cast<State*>(h);
  const unsigned n = st->nqubits;
  const uint64_t lim0 = n >= 64 ? ~0ull : ((1ull << n) - 1);
  const uint64_t lim1 = n <= 64 ? 0ull : ((1ull << (n - 64)) - 1);
  for (int w = 0; w < 2; ++w) {
    const uint64_t lim = w ? lim1 : lim0;
    if ((x[w] | z[w] | c[w]) & ~lim) return 1;
    if (c[w] & (x[w] | z[w])) return 1;
  }
  if ((x[0] | x[1] | z[0] | z[1]) == 0) return 1;
  const int ny = __builtin_popcountll(x[0] & z[0]) + __builtin_popcountll(x[1] & z[1]);
  const double cs = std::cos(0.5 * theta), sn = std::sin(0.5 * theta);
  Map out;
  out.reserve(2 * st->map.size());
  for (const auto& kv : st->map) {
    const Key& k = kv.first;
    const Cplx a = kv.second;
    if ((k.lo & c[0]) != c[0] || (k.hi & c[1]) != c[1]) {
      out[k] = cadd(out[k], a);
      continue;
    }
    // -i * i^nY * (-1)^parity = i^(nY + 3 + 2 parity)
    const int par = __builtin_popcountll(k.lo & z[0]) + __builtin_popcountll(k.hi & z[1]);
    const int e = (ny + 3 + 2 * par) & 3;
    const Cplx unit = e == 0 ? Cplx{1, 0} : e == 1 ? Cplx{0, 1} : e == 2 ? Cplx{-1, 0} : Cplx{0, -1};
    const Cplx w = Cplx{sn * unit.re, sn * unit.im};
    out[k] = cadd(out[k], Cplx{cs * a.re, cs * a.im});
    const Key kx{k.lo ^ x[0], k.hi ^ x[1]};
    out[kx] = cadd(out[kx], cmul(w, a));
  }
  prune(out, eps);
  st->map.swap(out);
  return 0;
}

// Measurement of qubit q in the computational basis with collapse (Sec. 2.1: the
// outcome b is observed with probability |alpha|^2 summed over the labels that
// show it, and the state is projected onto those labels; Sec. 3 lists
// measurements among the operations). Steps, in this order:
//   p0 = sum |alpha_k|^2 over labels with bit q = 0, p1 likewise for bit q = 1;
//   outcome = 1 iff r * (p0 + p1) < p1 (r in [0, 1) drawn by the caller);
//   the labels with bit q != outcome are removed and each kept amplitude is
//   divided by sqrt(p_outcome), so the state has norm 1 afterwards.
// out[0] = outcome, out[1] = p_outcome / (p0 + p1). Returns 1 on a bad
// argument, 0 otherwise; an empty state stays empty (outcome 0, probability 0).
int orc_measure(void* h, uint32_t q, double r, double* out) {
  State* st = static_cast<State*>(h);
  if (q >= st->nqubits || !(r >= 0.0 && r < 1.0)) return 1;
  const uint64_t bit = 1ull << (q & 63);
  double p0 = 0.0, p1 = 0.0;
  for (const auto& kv : st->map) {
    const uint64_t w = q < 64 ? kv.first.lo : kv.first.hi;
    const double m = kv.second.re * kv.second.re + kv.second.im * kv.second.im;
    if (w & bit) p1 += m; else p0 += m;
  }
  const double total = p0 + p1;
  const int outcome = r * total < p1 ? 1 : 0;
  const double pk = outcome ? p1 : p0;
  out[0] = outcome;
  out[1] = total > 0.0 ? pk / total : 0.0;
  Map m;
  if (pk > 0.0) {
    const double scale = 1.0 / std::sqrt(pk);
    for (const auto& kv : st->map) {
      const uint64_t w = q < 64 ? kv.first.lo : kv.first.hi;
      if (((w & bit) != 0) == (outcome == 1))
        m[kv.first] = Cplx{kv.second.re * scale, kv.second.im * scale};
    }
  }
  st->map.swap(m);
  return 0;
}

// ---- dense statevector checker (Sec. 2.2) -----------------------------------
// Runs the gates on |0...0> over all 2^n amplitudes. Only qubits < 64 and
// controls in word 0 are allowed (n <= 26). Returns 1 on a bad record.
int orc_dense_run(uint32_t n, const void* gates, uint64_t ngates, double* re, double* im) {
  if (n < 1 || n > 26) return 1;
  const uint64_t dim = 1ull << n;
  std::vector<std::complex<double>> v(dim, {0.0, 0.0});
  v[0] = {1.0, 0.0};
  const GateRec* gs = static_cast<const GateRec*>(gates);
  const double r = std::sqrt(0.5);
  for (uint64_t gi = 0; gi < ngates; ++gi) {
    const GateRec& g = gs[gi];
    if (!valid(g, n) || g.cmask[1] != 0) return 1;
    const uint64_t cm = g.cmask[0];
    const uint64_t tm = 1ull << g.t0;
    // 2x2 matrix U of the single-qubit gate, or the Givens block.
    std::complex<double> U[2][2];
    const double c = std::cos(0.5 * g.theta), s = std::sin(0.5 * g.theta);
    const std::complex<double> I(0.0, 1.0);
    switch (g.op) {
      case OP_X: U[0][0] = 0; U[0][1] = 1; U[1][0] = 1; U[1][1] = 0; break;
      case OP_Y: U[0][0] = 0; U[0][1] = -I; U[1][0] = I; U[1][1] = 0; break;
      case OP_Z: U[0][0] = 1; U[0][1] = 0; U[1][0] = 0; U[1][1] = -1.0; break;
      case OP_S: U[0][0] = 1; U[0][1] = 0; U[1][0] = 0; U[1][1] = I; break;
      case OP_SDG: U[0][0] = 1; U[0][1] = 0; U[1][0] = 0; U[1][1] = -I; break;
      case OP_T: U[0][0] = 1; U[0][1] = 0; U[1][0] = 0; U[1][1] = std::complex<double>(r, r); break;
      case OP_TDG: U[0][0] = 1; U[0][1] = 0; U[1][0] = 0; U[1][1] = std::complex<double>(r, -r); break;
      case OP_P:
        U[0][0] = 1; U[0][1] = 0; U[1][0] = 0;
        U[1][1] = std::complex<double>(std::cos(g.theta), std::sin(g.theta));
        break;
      case OP_RZ:
        U[0][0] = std::complex<double>(c, -s); U[0][1] = 0; U[1][0] = 0;
        U[1][1] = std::complex<double>(c, s);
        break;
      case OP_H: U[0][0] = r; U[0][1] = r; U[1][0] = r; U[1][1] = -r; break;
      case OP_RX: U[0][0] = c; U[0][1] = -I * s; U[1][0] = -I * s; U[1][1] = c; break;
      case OP_RY: U[0][0] = c; U[0][1] = -s; U[1][0] = s; U[1][1] = c; break;
      case OP_GIVENS:
        U[0][0] = std::cos(g.theta); U[0][1] = -std::sin(g.theta);
        U[1][0] = std::sin(g.theta); U[1][1] = std::cos(g.theta);
        break;
      default: return 1;
    }
    if (g.op == OP_GIVENS) {
      const uint64_t pm = 1ull << g.t0, qm = 1ull << g.t1;
      for (uint64_t i = 0; i < dim; ++i) {
        // i is the (p=0, q=1) member of its pair
        if ((i & pm) || !(i & qm) || (i & cm) != cm) continue;
        const uint64_t j = (i | pm) & ~qm;
        const std::complex<double> a0 = v[i], a1 = v[j];
        v[i] = U[0][0] * a0 + U[0][1] * a1;
        v[j] = U[1][0] * a0 + U[1][1] * a1;
      }
    } else {
      for (uint64_t i = 0; i < dim; ++i) {
        if ((i & tm) || (i & cm) != cm) continue;
        const uint64_t j = i | tm;
        const std::complex<double> a0 = v[i], a1 = v[j];
        v[i] = U[0][0] * a0 + U[0][1] * a1;
        v[j] = U[1][0] * a0 + U[1][1] * a1;
      }
    }
  }
  for (uint64_t i = 0; i < dim; ++i) {
    re[i] = v[i].real();
    im[i] = v[i].imag();
  }
  return 0;
}

// ---- classical evaluator for permutation-only circuits ----------------------
// Pushes each key through the X gates (any number of controls) in order.
// Returns 1 with *bad set if a record is not an X gate or is invalid.
int orc_classical_eval(uint32_t n, const void* gates, uint64_t ngates, uint64_t* hi,
                       uint64_t* lo, uint64_t nkeys, uint64_t* bad) {
  const GateRec* gs = static_cast<const GateRec*>(gates);
  for (uint64_t gi = 0; gi < ngates; ++gi) {
    if (gs[gi].op != OP_X || !valid(gs[gi], n)) {
      if (bad) *bad = gi;
      return 1;
    }
  }
  for (uint64_t i = 0; i < nkeys; ++i) {
    Key k{lo[i], hi[i]};
    for (uint64_t gi = 0; gi < ngates; ++gi) {
      if (controls_hold(k, gs[gi])) k = flip(k, gs[gi].t0);
    }
    lo[i] = k.lo;
    hi[i] = k.hi;
  }
  return 0;
}

}  // extern "C"

// ---- dense simulator on a fixed-weight sector ---------------------------------
// Gates that conserve the number of set bits (Givens, and the diagonal gates
// Z, S, Sdg, T, Tdg, P, Rz with any controls) keep a state inside the span of
// the C(n, k) labels of weight k. This checker holds ALL of them as a dense
// vector, one amplitude per label, indexed by the combinatorial number system
// (colex rank: for set bits c_1 < ... < c_k the index is sum_i C(c_i, i)).
// Gosper's successor enumerates the labels in increasing order, which is the
// same order, so label[rank] is filled by counting. No pruning, no map: a
// pair (i, j) of a Givens gate is found by ranking the partner label.
// The arithmetic of each amplitude is the same as the sparse simulator's
// (the same complex products and sums, in the same order), so without pruning
// the two agree bit for bit. n <= 64 (labels in one word).
namespace {
uint64_t binom_tab[65][65];
bool binom_ready = false;
void binom_init() {
  if (binom_ready) return;
  for (int a = 0; a <= 64; ++a) {
    binom_tab[a][0] = 1;
    for (int b = 1; b <= 64; ++b)
      binom_tab[a][b] = a == 0 ? 0 : binom_tab[a - 1][b - 1] + binom_tab[a - 1][b];
  }
  binom_ready = true;
}
uint64_t colex_rank(uint64_t label) {
  uint64_t r = 0;
  int i = 1;
  while (label) {
    const int c = __builtin_ctzll(label);
    r += binom_tab[c][i];
    ++i;
    label &= label - 1;
  }
  return r;
}
bool sector_gate_ok(const GateRec& g) {
  switch (g.op) {
    case OP_GIVENS: case OP_Z: case OP_S: case OP_SDG: case OP_T: case OP_TDG:
    case OP_P: case OP_RZ:
      return true;
    default:
      return false;
  }
}
}  // namespace

extern "C" {

// Number of labels of the sector of `start` on n qubits (C(n, popcount)).
uint64_t orc_sector_size(uint32_t n, uint64_t start) {
  binom_init();
  if (n < 1 || n > 64) return 0;
  return binom_tab[n][__builtin_popcountll(start)];
}

// Runs the gates on |start> inside its weight sector. labels/re/im receive
// all C(n, k) labels (increasing) and their amplitudes (zeros included).
// Returns 0, 1 on an invalid record or one that leaves the sector (*bad set),
// 2 if cap < C(n, k) or n is out of range.
int orc_sector_run(uint32_t n, uint64_t start, const void* gates, uint64_t ngates,
                   uint64_t* labels, double* re, double* im, uint64_t cap, uint64_t* bad) {
  binom_init();
  if (n < 1 || n > 64) return 2;
  if (n < 64 && (start >> n) != 0) return 2;
  const int k = __builtin_popcountll(start);
  const uint64_t size = binom_tab[n][k];
  if (cap < size) return 2;
  const GateRec* gs = static_cast<const GateRec*>(gates);
  for (uint64_t gi = 0; gi < ngates; ++gi) {
    if (!valid(gs[gi], n) || !sector_gate_ok(gs[gi]) || gs[gi].cmask[1] != 0) {
      if (bad) *bad = gi;
      return 1;
    }
  }
  // labels of weight k in increasing order (Gosper's successor)
  uint64_t v = k == 0 ? 0ull : (k == 64 ? ~0ull : ((1ull << k) - 1));
  for (uint64_t r = 0; r < size; ++r) {
    labels[r] = v;
    if (r + 1 < size) {
      const uint64_t t = v | (v - 1);
      v = (t + 1) | (((~t & -~t) - 1) >> (__builtin_ctzll(v) + 1));
    }
  }
  std::vector<Cplx> a(size, Cplx{0.0, 0.0});
  a[colex_rank(start)] = Cplx{1.0, 0.0};
  for (uint64_t gi = 0; gi < ngates; ++gi) {
    const GateRec& g = gs[gi];
    const uint64_t cm = g.cmask[0];
    if (g.op == OP_GIVENS) {
      Cplx M[2][2];
      branch_matrix(g, M);
      const uint64_t pm = 1ull << g.t0, qm = 1ull << g.t1;
      for (uint64_t r = 0; r < size; ++r) {
        const uint64_t L = labels[r];
        // r is the first member of its pair: bit p = 0, bit q = 1
        if ((L & pm) || !(L & qm) || (L & cm) != cm) continue;
        const uint64_t j = colex_rank((L | pm) & ~qm);
        const Cplx a0 = a[r], a1 = a[j];
        a[r] = cadd(cmul(M[0][0], a0), cmul(M[0][1], a1));
        a[j] = cadd(cmul(M[1][0], a0), cmul(M[1][1], a1));
      }
    } else {
      // the factor on a label whose controls hold, by its target bit (taken
      // from the gate's definition once per gate); elsewhere the factor is 1
      Key same;
      const Key k0{cm, 0ull};
      const Key k1{cm | (1ull << g.t0), 0ull};
      const Cplx f0 = perm_diag_action(g, k0, &same);
      const Cplx f1 = perm_diag_action(g, k1, &same);
      const uint64_t tm = 1ull << g.t0;
      for (uint64_t r = 0; r < size; ++r) {
        const uint64_t L = labels[r];
        if ((L & cm) != cm) continue;
        const Cplx f = (L & tm) ? f1 : f0;
        if (f.re == 1.0 && f.im == 0.0) continue;   // 1 * a = a
        a[r] = cmul(f, a[r]);
      }
    }
  }
  for (uint64_t r = 0; r < size; ++r) {
    re[r] = a[r].re;
    im[r] = a[r].im;
  }
  return 0;
}

}  // extern "C"
