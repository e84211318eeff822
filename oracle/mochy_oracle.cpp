// Reference oracle for MoCHy h-motif / 3h-motif counting.
//
// TEST INFRASTRUCTURE ONLY.  This file is a plain, slow CPU restatement of
// the paper's definitions and algorithms ("Hypergraph motifs and their
// extensions beyond binary", arXiv 2310.15668).  Only the test suite, the
// smoke check and the bench's CPU-baseline leg may load it.  It shares no
// code, header, table or constant generator with the CUDA library; the two
// are checked against each other.  Everything runs on one thread except the
// anchor loop of orc_count_exact_ranked and orc_line_degrees, which may
// share their outer loop among host threads (the paper's own parallel
// scheme, each thread with its own histogram).
//
// Every function cites the passage it follows.  Hash containers are the
// standard library's, as in the paper's own implementation (Section 5.1).
//
// Readings of the paper where it is silent or garbled (each also listed in
// the design notes):
//   R1  h-motif numbering (the figure that fixes it is lost): canonical
//       pattern = lexicographically smallest region tuple (1)..(7) over the
//       six role permutations (Appendix "Extensions beyond Three Hyperedges",
//       the P_1 rule); ids 1-16 = closed with a non-empty triple region,
//       17-22 = open, 23-26 = closed with an empty triple region, each group
//       in ascending canonical tuple order.
//   R2  3h-motif numbering (figure lost): ascending (h-motif id, canonical
//       ternary tuple).
//   R3  theta = 1: states 0, 1, >=2 (Section 4.1).
//   R4  A+ rescaling follows Algorithm "sampling_ver2" and Eq. (w[t]):
//       open w = 2, closed w = 3 (the footnote that swaps them is a typo).
//   R5  randomized copies: Chung-Lu draws (Algorithm "randomized_hypergraph_
//       alg"), sets per hyperedge, empty ones dropped (Algorithm "transform"),
//       then duplicate hyperedges dropped keeping the first, because E is a
//       set (Section 2.1 footnote).
//   R6  random draws: Philox4x32-10 (Salmon et al., SC'11); a 64-bit uniform
//       u is mapped to [0, n) as floor(u * n / 2^64).
//   R7  sample n of a sampling run uses counter (n_lo, n_hi, stream, 0) and
//       key (seed_lo, seed_hi); hyperwedges are indexed in ascending (i, j)
//       order with i < j.
//   R8  estimates are (double)raw * (double)scale_num / ((double)w *
//       (double)samples), no fused multiply-add.
//   R9  M_rand is the mean over the copies; eps = 1; a CP whose significances
//       are all zero is returned as zeros.
//   R10 hyperedge ids are positions after duplicate removal (first
//       occurrence kept, input order preserved).
//   R11 in the variance theorems of MoCHy-A / MoCHy-A+, p_l[t] and q_n[t]
//       count ordered pairs of distinct instances (the reading under which
//       the stated formulas are the estimators' variances).
//   R12 node profiles: the star ego-network of v keeps the hyperedges that
//       contain v whole, and its instances are classified as in G.
//
// Parity pins: see tests/test_oracle_*.py (motif-table counts printed in the
// paper, brute force over all triples, invariants, Philox known answers,
// closed forms of the estimators and of the Chung-Lu expectations, the
// per-anchor sampling bodies and the variance theorems, brute force of the
// hyperedge and star node profiles).  The motif numbering's agreement with
// the paper's lost figures (R1, R2) is unpinned: the tests compare patterns.

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <mutex>
#include <set>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

// ---------------------------------------------------------------------------
// Motif tables (Section 2.2 "Definition and Representation", Section 4.1,
// Appendix "Extensions beyond Three Hyperedges").
// ---------------------------------------------------------------------------

// A pattern is a 7-tuple of region states in the paper's region order:
// (1) i\j\k (2) j\k\i (3) k\i\j (4) i&j\k (5) j&k\i (6) k&i\j (7) i&j&k.
using Pattern = std::array<int, 7>;

// Region index of each non-empty subset of the three roles {i=0, j=1, k=2}.
int region_of_subset(int mask) {
  switch (mask) {
    case 1: return 0;   // {i}
    case 2: return 1;   // {j}
    case 4: return 2;   // {k}
    case 3: return 3;   // {i,j}
    case 6: return 4;   // {j,k}
    case 5: return 5;   // {k,i}
    case 7: return 6;   // {i,j,k}
  }
  return -1;
}

// Re-label the three roles by the permutation perm (role r -> perm[r]).
Pattern permute(const Pattern& p, const int perm[3]) {
  Pattern q{};
  for (int s = 1; s < 8; ++s) {
    int t = 0;
    for (int r = 0; r < 3; ++r)
      if (s & (1 << r)) t |= 1 << perm[r];
    q[region_of_subset(t)] = p[region_of_subset(s)];
  }
  return q;
}

const int kPerms[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2},
                          {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

// Lexicographically smallest tuple over the six permutations (P_1 rule).
Pattern canonical(const Pattern& p) {
  Pattern best = p;
  for (auto& perm : kPerms) {
    Pattern q = permute(p, perm);
    if (q < best) best = q;
  }
  return best;
}

// Pairs {i,j}: regions (4) and (7); {j,k}: (5),(7); {k,i}: (6),(7).
bool pair_meets(const Pattern& p, int pair) {
  const int reg[3] = {3, 4, 5};
  return p[reg[pair]] > 0 || p[6] > 0;
}

// Connected (Section 2.1): some hyperedge is adjacent to the other two, i.e.
// at least two of the three pairs intersect.
bool connected(const Pattern& p) {
  int n = 0;
  for (int q = 0; q < 3; ++q) n += pair_meets(p, q) ? 1 : 0;
  return n >= 2;
}

bool closed_pattern(const Pattern& p) {
  return pair_meets(p, 0) && pair_meets(p, 1) && pair_meets(p, 2);
}

// Distinct hyperedges (Fig. "motif_three_hyperedges_duplicated"): e_x = e_y
// exactly when both regions that hold x but not y and both that hold y but
// not x are empty.
bool distinct(const Pattern& p) {
  // e_i \ e_j = (1) u (6); e_j \ e_i = (2) u (5)
  // e_j \ e_k = (2) u (4); e_k \ e_j = (3) u (6)
  // e_k \ e_i = (3) u (5); e_i \ e_k = (1) u (4)
  auto empty2 = [&](int a, int b) { return p[a] == 0 && p[b] == 0; };
  if (empty2(0, 5) && empty2(1, 4)) return false;
  if (empty2(1, 3) && empty2(2, 5)) return false;
  if (empty2(2, 4) && empty2(0, 3)) return false;
  return true;
}

struct Tables {
  // lut_h[code] with code = sum_p [region p non-empty] << p  -> id 1..26 or 0
  std::array<int32_t, 128> lut_h{};
  // lut_3h[code] with code = sum_p state_p * 3^p            -> id 1..431 or 0
  std::array<int32_t, 2187> lut_3h{};
  std::vector<Pattern> h_pattern;   // index id-1
  std::vector<Pattern> t_pattern;   // index id-1
  std::vector<int32_t> t_to_h;      // index id-1 -> h id
  std::vector<uint8_t> h_open;      // index id-1
  // stats of the filtering chain (Table "hmotif_cnt_table", Section 4.1)
  int64_t n_all = 0, n_unique = 0, n_connected = 0, n_valid = 0;
  int64_t t_all = 0, t_unique = 0, t_connected = 0, t_valid = 0;
};

int h_group(const Pattern& p) {
  if (!closed_pattern(p)) return 1;   // open: ids 17-22
  return p[6] > 0 ? 0 : 2;            // closed with / without triple region
}

Tables build_tables() {
  Tables T;
  // Binary patterns.
  std::set<Pattern> uniq, conn, valid;
  for (int code = 0; code < 128; ++code) {
    Pattern p{};
    for (int r = 0; r < 7; ++r) p[r] = (code >> r) & 1;
    Pattern c = canonical(p);
    uniq.insert(c);
    if (connected(c)) conn.insert(c);
    if (connected(c) && distinct(c)) valid.insert(c);
  }
  T.n_all = 128;
  T.n_unique = (int64_t)uniq.size();
  T.n_connected = (int64_t)conn.size();
  T.n_valid = (int64_t)valid.size();
  std::vector<std::pair<std::pair<int, Pattern>, Pattern>> order;
  for (auto& c : valid) order.push_back({{h_group(c), c}, c});
  std::sort(order.begin(), order.end());
  std::map<Pattern, int> h_id;
  for (size_t n = 0; n < order.size(); ++n) {
    h_id[order[n].second] = (int)n + 1;
    T.h_pattern.push_back(order[n].second);
    T.h_open.push_back(closed_pattern(order[n].second) ? 0 : 1);
  }
  for (int code = 0; code < 128; ++code) {
    Pattern p{};
    for (int r = 0; r < 7; ++r) p[r] = (code >> r) & 1;
    Pattern c = canonical(p);
    auto it = h_id.find(c);
    T.lut_h[code] = it == h_id.end() ? 0 : it->second;
  }
  // Ternary patterns (theta = 1: states 0, 1, 2 = ">1").
  std::set<Pattern> tu, tc, tv;
  for (int code = 0; code < 2187; ++code) {
    Pattern p{};
    int x = code;
    for (int r = 0; r < 7; ++r) { p[r] = x % 3; x /= 3; }
    Pattern c = canonical(p);
    tu.insert(c);
    if (connected(c)) tc.insert(c);
    if (connected(c) && distinct(c)) tv.insert(c);
  }
  T.t_all = 2187;
  T.t_unique = (int64_t)tu.size();
  T.t_connected = (int64_t)tc.size();
  T.t_valid = (int64_t)tv.size();
  std::vector<std::pair<std::pair<int, Pattern>, Pattern>> torder;
  for (auto& c : tv) {
    Pattern b{};
    for (int r = 0; r < 7; ++r) b[r] = c[r] > 0 ? 1 : 0;
    int hid = h_id.at(canonical(b));
    torder.push_back({{hid, c}, c});
  }
  std::sort(torder.begin(), torder.end());
  std::map<Pattern, int> t_id;
  for (size_t n = 0; n < torder.size(); ++n) {
    t_id[torder[n].second] = (int)n + 1;
    T.t_pattern.push_back(torder[n].second);
    T.t_to_h.push_back(torder[n].first.first);
  }
  for (int code = 0; code < 2187; ++code) {
    Pattern p{};
    int x = code;
    for (int r = 0; r < 7; ++r) { p[r] = x % 3; x /= 3; }
    auto it = t_id.find(canonical(p));
    T.lut_3h[code] = it == t_id.end() ? 0 : it->second;
  }
  return T;
}

const Tables& tables() {
  static const Tables T = build_tables();
  return T;
}

// kh-motifs (Section 4.1 "Extensions Beyond Ternary"): each region takes one
// of k states, 0 for empty and s for a cardinality c with
// thr[s-2] < c <= thr[s-1] (thr[-1] = 0, thr[k-2] = infinity).  Patterns are
// canonicalised, filtered and numbered as the 3h-motifs are (readings R1,
// R2: ascending (h-motif id, canonical tuple)).
struct KTables {
  int k = 0;
  std::vector<int32_t> lut;        // k^7 codes (digit p has weight k^p) -> id or 0
  std::vector<Pattern> pattern;    // index id-1
  std::vector<int32_t> to_h;       // index id-1 -> h id
};

KTables build_k_tables(int k) {
  const Tables& T = tables();
  KTables K;
  K.k = k;
  int64_t total = 1;
  for (int r = 0; r < 7; ++r) total *= k;
  auto decode = [&](int64_t code) {
    Pattern p{};
    for (int r = 0; r < 7; ++r) { p[r] = (int)(code % k); code /= k; }
    return p;
  };
  std::set<Pattern> valid;
  for (int64_t code = 0; code < total; ++code) {
    Pattern c = canonical(decode(code));
    if (connected(c) && distinct(c)) valid.insert(c);
  }
  auto parent = [&](const Pattern& c) {
    int b = 0;
    for (int r = 0; r < 7; ++r) b |= (c[r] > 0 ? 1 : 0) << r;
    return T.lut_h[b];
  };
  std::vector<std::pair<std::pair<int, Pattern>, Pattern>> order;
  for (auto& c : valid) order.push_back({{parent(c), c}, c});
  std::sort(order.begin(), order.end());
  std::map<Pattern, int> id;
  for (size_t n = 0; n < order.size(); ++n) {
    id[order[n].second] = (int)n + 1;
    K.pattern.push_back(order[n].second);
    K.to_h.push_back(order[n].first.first);
  }
  K.lut.assign((size_t)total, 0);
  for (int64_t code = 0; code < total; ++code) {
    auto it = id.find(canonical(decode(code)));
    K.lut[(size_t)code] = it == id.end() ? 0 : it->second;
  }
  return K;
}

const KTables& k_tables(int k) {
  static std::map<int, KTables> cache;
  static std::mutex mu;
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(k);
  if (it == cache.end()) it = cache.emplace(k, build_k_tables(k)).first;
  return it->second;
}

// state of a region of cardinality c among k states with the k - 2
// ascending thresholds thr: 0 when empty, else 1 + the number exceeded
int k_state(int64_t c, int k, const int32_t* thr) {
  if (c == 0) return 0;
  int s = 1;
  for (int m = 0; m < k - 2; ++m) s += c > thr[m] ? 1 : 0;
  return s;
}

// ---------------------------------------------------------------------------
// Hypergraph (Section 2.1).  E is a set of non-empty node sets.
// ---------------------------------------------------------------------------

struct Hypergraph {
  std::vector<std::vector<int32_t>> e;                 // sorted node lists
  std::vector<std::unordered_set<int32_t>> eset;       // same, as hash sets
  std::unordered_map<int32_t, std::vector<int32_t>> ev; // E_v
};

// Sort node lists, reject empty hyperedges, drop duplicates keeping the
// first occurrence (Section 2.1 footnote; reading R10).
int load(int64_t n_edges, const int64_t* off, const int32_t* nodes,
         Hypergraph& G, int64_t* n_dup) {
  std::set<std::vector<int32_t>> seen;
  int64_t dup = 0;
  for (int64_t i = 0; i < n_edges; ++i) {
    if (off[i + 1] <= off[i]) return -1;
    std::vector<int32_t> s(nodes + off[i], nodes + off[i + 1]);
    std::sort(s.begin(), s.end());
    s.erase(std::unique(s.begin(), s.end()), s.end());
    if (s.front() < 0) return -1;
    if (!seen.insert(s).second) { ++dup; continue; }
    G.e.push_back(s);
  }
  for (size_t i = 0; i < G.e.size(); ++i) {
    G.eset.emplace_back(G.e[i].begin(), G.e[i].end());
    for (int32_t v : G.e[i]) G.ev[v].push_back((int32_t)i);
  }
  if (n_dup) *n_dup = dup;
  return 0;
}

uint64_t pair_key(int64_t i, int64_t j) {
  if (i > j) std::swap(i, j);
  return ((uint64_t)i << 32) | (uint64_t)j;
}

// Algorithm "hyperwedge_counting" (line-graph construction, Section 3.1):
// for each e_i, each v in e_i, each e_j in E_v with j > i: add the
// hyperwedge and increment omega.
struct LineGraph {
  std::unordered_map<uint64_t, int32_t> omega;
  std::vector<std::vector<int32_t>> nbr;   // N_{e_i}
};

LineGraph project(const Hypergraph& G) {
  LineGraph L;
  const int64_t E = (int64_t)G.e.size();
  for (int64_t i = 0; i < E; ++i)
    for (int32_t v : G.e[i])
      for (int32_t j : G.ev.at(v))
        if (j > i) L.omega[pair_key(i, j)] += 1;
  L.nbr.assign(E, {});
  for (auto& kv : L.omega) {
    int32_t i = (int32_t)(kv.first >> 32), j = (int32_t)(kv.first & 0xffffffffu);
    L.nbr[i].push_back(j);
    L.nbr[j].push_back(i);
  }
  for (auto& n : L.nbr) std::sort(n.begin(), n.end());
  return L;
}

int32_t omega_of(const LineGraph& L, int64_t i, int64_t j) {
  auto it = L.omega.find(pair_key(i, j));
  return it == L.omega.end() ? 0 : it->second;
}

// Lemma "motif:time": the seven region cardinalities of {e_i, e_j, e_k} from
// the three sizes, the three overlaps and |e_i & e_j & e_k|, the latter
// found by checking each node of the smallest hyperedge against the other
// two hash sets.
std::array<int64_t, 7> regions(const Hypergraph& G, int64_t i, int64_t j,
                               int64_t k, int64_t wij, int64_t wjk,
                               int64_t wki) {
  int64_t a = i, b = j, c = k;
  if (G.e[b].size() < G.e[a].size()) std::swap(a, b);
  if (G.e[c].size() < G.e[a].size()) std::swap(a, c);
  int64_t t = 0;
  for (int32_t v : G.e[a])
    if (G.eset[b].count(v) && G.eset[c].count(v)) ++t;
  const int64_t si = (int64_t)G.e[i].size(), sj = (int64_t)G.e[j].size(),
                sk = (int64_t)G.e[k].size();
  return {si - wij - wki + t, sj - wij - wjk + t, sk - wki - wjk + t,
          wij - t, wjk - t, wki - t, t};
}

// h(.) and h3(.) (Section 2.2; Section 4.1 with theta from R3).
void classify(const std::array<int64_t, 7>& r, int32_t theta, int* h, int* h3) {
  const Tables& T = tables();
  int code2 = 0, code3 = 0, pw = 1;
  for (int p = 0; p < 7; ++p) {
    code2 |= (r[p] > 0 ? 1 : 0) << p;
    int st = r[p] == 0 ? 0 : (r[p] <= theta ? 1 : 2);
    code3 += st * pw;
    pw *= 3;
  }
  *h = T.lut_h[code2];
  *h3 = T.lut_3h[code3];
}

// Algorithm "exact_motif_counting" (MoCHy-E): for each e_i, each unordered
// pair {e_j, e_k} of its neighbours, count it when e_j and e_k are disjoint
// or i < min(j, k).  Restricted to the anchors in `only` when non-null.
// With hp_h / hp_3h (|E| x 26 / |E| x 431, may be null) every counted
// instance is also added to the rows of its three hyperedges: the hyperedge
// profile (Section 3.1, "Hyperedge Profile (HP)": the t-th element of HP(e)
// is the number of instances of motif t that include e).
void exact_count(const Hypergraph& G, const LineGraph& L, int32_t theta,
                 const std::vector<int32_t>* only, int64_t* out_h,
                 int64_t* out_3h, int64_t* hp_h = nullptr, int64_t* hp_3h = nullptr) {
  std::fill(out_h, out_h + 26, 0);
  std::fill(out_3h, out_3h + 431, 0);
  const int64_t E = (int64_t)G.e.size();
  std::vector<int32_t> all;
  if (!only) {
    all.resize(E);
    for (int64_t i = 0; i < E; ++i) all[i] = (int32_t)i;
    only = &all;
  }
  for (int32_t i : *only) {
    const auto& N = L.nbr[i];
    for (size_t x = 0; x < N.size(); ++x)
      for (size_t y = x + 1; y < N.size(); ++y) {
        const int32_t j = N[x], k = N[y];
        const int32_t wjk = omega_of(L, j, k);
        if (!(wjk == 0 || i < std::min(j, k))) continue;
        auto r = regions(G, i, j, k, omega_of(L, i, j), wjk, omega_of(L, k, i));
        int h, h3;
        classify(r, theta, &h, &h3);
        out_h[h - 1] += 1;
        out_3h[h3 - 1] += 1;
        for (int32_t e : {i, j, k}) {
          if (hp_h) hp_h[(int64_t)e * 26 + h - 1] += 1;
          if (hp_3h) hp_3h[(int64_t)e * 431 + h3 - 1] += 1;
        }
      }
  }
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
// easy as 1, 2, 3", SC'11), written from its published description.
// ---------------------------------------------------------------------------

struct U4 { uint32_t v[4]; };

U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += W0; k1 += W1; }
    const uint64_t p0 = (uint64_t)M0 * c.v[0];
    const uint64_t p1 = (uint64_t)M1 * c.v[2];
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    U4 n;
    n.v[0] = hi1 ^ c.v[1] ^ k0;
    n.v[1] = lo1;
    n.v[2] = hi0 ^ c.v[3] ^ k1;
    n.v[3] = lo0;
    c = n;
  }
  return c;
}

// 64-bit uniform of draw (a, b) in stream s under seed (reading R6/R7).
uint64_t draw_u64(uint64_t seed, uint64_t n, uint32_t stream, uint32_t extra) {
  U4 c{{(uint32_t)n, (uint32_t)(n >> 32), stream, extra}};
  U4 o = philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
  return ((uint64_t)o.v[1] << 32) | o.v[0];
}

uint64_t scale_index(uint64_t u, uint64_t n) {
  return (uint64_t)(((unsigned __int128)u * n) >> 64);
}

const uint32_t kStreamEdgeSample = 1;    // MoCHy-A hyperedge samples
const uint32_t kStreamWedgeSample = 2;   // MoCHy-A+ hyperwedge samples
const uint32_t kStreamChungLuNode = 3;   // Chung-Lu node endpoint
const uint32_t kStreamChungLuEdge = 4;   // Chung-Lu hyperedge endpoint

// All hyperwedges in ascending (i, j) order, i < j (reading R7).
std::vector<std::pair<int32_t, int32_t>> sorted_wedges(const LineGraph& L) {
  std::vector<std::pair<int32_t, int32_t>> w;
  w.reserve(L.omega.size());
  for (auto& kv : L.omega)
    w.push_back({(int32_t)(kv.first >> 32), (int32_t)(kv.first & 0xffffffffu)});
  std::sort(w.begin(), w.end());
  return w;
}

void add_instance(const Hypergraph& G, const LineGraph& L, int32_t theta,
                  int64_t i, int64_t j, int64_t k, int64_t* raw_h,
                  int64_t* raw_3h) {
  auto r = regions(G, i, j, k, omega_of(L, i, j), omega_of(L, j, k),
                   omega_of(L, k, i));
  int h, h3;
  classify(r, theta, &h, &h3);
  raw_h[h - 1] += 1;
  raw_3h[h3 - 1] += 1;
}

// Algorithm "sampling_ver1" (MoCHy-A): s hyperedges uniformly with
// replacement; every instance containing the sample is counted once (k not
// a neighbour of e_i, or j < k).
void count_A(const Hypergraph& G, const LineGraph& L, int32_t theta,
             int64_t s, uint64_t seed, int64_t* raw_h, int64_t* raw_3h) {
  const uint64_t E = G.e.size();
  for (int64_t n = 0; n < s; ++n) {
    const int64_t i = (int64_t)scale_index(draw_u64(seed, n, kStreamEdgeSample, 0), E);
    const auto& Ni = L.nbr[i];
    std::unordered_set<int32_t> inNi(Ni.begin(), Ni.end());
    for (int32_t j : Ni) {
      std::set<int32_t> cand(Ni.begin(), Ni.end());
      cand.insert(L.nbr[j].begin(), L.nbr[j].end());
      cand.erase((int32_t)i);
      cand.erase(j);
      for (int32_t k : cand)
        if (!inNi.count(k) || j < k) add_instance(G, L, theta, i, j, k, raw_h, raw_3h);
    }
  }
}

// Algorithm "sampling_ver2" (MoCHy-A+): r hyperwedges uniformly with
// replacement; every e_k adjacent to e_i or e_j is counted.
void count_Aplus(const Hypergraph& G, const LineGraph& L, int32_t theta,
                 int64_t r, uint64_t seed, int64_t* raw_h, int64_t* raw_3h) {
  auto W = sorted_wedges(L);
  const uint64_t nw = W.size();
  for (int64_t n = 0; n < r; ++n) {
    auto w = W[scale_index(draw_u64(seed, n, kStreamWedgeSample, 0), nw)];
    const int32_t i = w.first, j = w.second;
    std::set<int32_t> cand(L.nbr[i].begin(), L.nbr[i].end());
    cand.insert(L.nbr[j].begin(), L.nbr[j].end());
    cand.erase(i);
    cand.erase(j);
    for (int32_t k : cand) add_instance(G, L, theta, i, j, k, raw_h, raw_3h);
  }
}

// Algorithms "randomized_hypergraph_alg" (Chung-Lu on the incidence graph)
// and "transform", with reading R5: |E'| draws of (node ~ degree,
// hyperedge ~ size); node sets per hyperedge; empty ones dropped;
// duplicates dropped keeping the first.
void randomize(const Hypergraph& G, int64_t n_nodes, uint64_t seed,
               uint32_t copy, std::vector<std::vector<int32_t>>& out) {
  const int64_t E = (int64_t)G.e.size();
  std::vector<int64_t> deg(n_nodes, 0);
  for (auto& e : G.e)
    for (int32_t v : e) deg[v] += 1;
  std::vector<int64_t> vpre(n_nodes + 1, 0), epre(E + 1, 0);
  for (int64_t v = 0; v < n_nodes; ++v) vpre[v + 1] = vpre[v] + deg[v];
  for (int64_t j = 0; j < E; ++j) epre[j + 1] = epre[j] + (int64_t)G.e[j].size();
  const int64_t total = epre[E];
  std::vector<std::set<int32_t>> ehat(E);
  for (int64_t d = 0; d < total; ++d) {
    const uint64_t xv = scale_index(draw_u64(seed, d, kStreamChungLuNode, copy), total);
    const uint64_t xe = scale_index(draw_u64(seed, d, kStreamChungLuEdge, copy), total);
    // the node v with vpre[v] <= x < vpre[v+1]
    const int64_t v = (int64_t)(std::upper_bound(vpre.begin(), vpre.end(), (int64_t)xv) - vpre.begin()) - 1;
    const int64_t j = (int64_t)(std::upper_bound(epre.begin(), epre.end(), (int64_t)xe) - epre.begin()) - 1;
    ehat[j].insert((int32_t)v);
  }
  std::set<std::vector<int32_t>> seen;
  out.clear();
  for (int64_t j = 0; j < E; ++j) {
    if (ehat[j].empty()) continue;
    std::vector<int32_t> s(ehat[j].begin(), ehat[j].end());
    if (seen.insert(s).second) out.push_back(s);
  }
}

// Eq. "significance" and Eq. "cp" (Section 3.1) in FP64 (reading R9).
void significance_cp(const int64_t* M, const double* Mrand, int n, double eps,
                     double* sig, double* cp, int* degenerate) {
  double ss = 0.0;
  for (int t = 0; t < n; ++t) {
    const double m = (double)M[t];
    sig[t] = (m - Mrand[t]) / (m + Mrand[t] + eps);
    ss += sig[t] * sig[t];
  }
  const double norm = std::sqrt(ss);
  *degenerate = norm == 0.0 ? 1 : 0;
  for (int t = 0; t < n; ++t) cp[t] = norm == 0.0 ? 0.0 : sig[t] / norm;
}

int build(int64_t n_edges, const int64_t* off, const int32_t* nodes,
          Hypergraph& G) {
  if (n_edges < 0 || !off) return -1;
  return load(n_edges, off, nodes, G, nullptr);
}

}  // namespace

// ---------------------------------------------------------------------------
// C entry points (loaded with ctypes by the tests).
// ---------------------------------------------------------------------------
extern "C" {

int orc_tables(int32_t* lut_h, int32_t* lut_3h, uint8_t* h_pattern,
               uint8_t* t_pattern, int32_t* t_to_h, uint8_t* h_open,
               int64_t* chain) {
  const Tables& T = tables();
  if (T.h_pattern.size() != 26 || T.t_pattern.size() != 431) return -2;
  std::memcpy(lut_h, T.lut_h.data(), sizeof(int32_t) * 128);
  std::memcpy(lut_3h, T.lut_3h.data(), sizeof(int32_t) * 2187);
  for (int n = 0; n < 26; ++n)
    for (int r = 0; r < 7; ++r) h_pattern[n * 7 + r] = (uint8_t)T.h_pattern[n][r];
  for (int n = 0; n < 431; ++n)
    for (int r = 0; r < 7; ++r) t_pattern[n * 7 + r] = (uint8_t)T.t_pattern[n][r];
  std::memcpy(t_to_h, T.t_to_h.data(), sizeof(int32_t) * 431);
  std::memcpy(h_open, T.h_open.data(), 26);
  const int64_t c[8] = {T.n_all, T.n_unique, T.n_connected, T.n_valid,
                        T.t_all, T.t_unique, T.t_connected, T.t_valid};
  std::memcpy(chain, c, sizeof(c));
  return 0;
}

// Canonical pattern chain for an arbitrary number of states per region
// (kh-motifs, Section 4.1 "Extensions Beyond Ternary"): returns the number
// of valid canonical patterns with k states.
int64_t orc_count_kh(int k) {
  int64_t total = 1;
  for (int r = 0; r < 7; ++r) total *= k;
  std::set<Pattern> valid;
  for (int64_t code = 0; code < total; ++code) {
    Pattern p{};
    int64_t x = code;
    for (int r = 0; r < 7; ++r) { p[r] = (int)(x % k); x /= k; }
    Pattern c = canonical(p);
    if (connected(c) && distinct(c)) valid.insert(c);
  }
  return (int64_t)valid.size();
}

int orc_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out) {
  U4 c{{ctr[0], ctr[1], ctr[2], ctr[3]}};
  U4 o = philox4x32_10(c, key[0], key[1]);
  std::memcpy(out, o.v, 16);
  return 0;
}

int orc_dedupe(int64_t n_edges, const int64_t* off, const int32_t* nodes,
               int64_t* out_off, int32_t* out_nodes, int64_t* n_out,
               int64_t* n_dup) {
  Hypergraph G;
  int rc = load(n_edges, off, nodes, G, n_dup);
  if (rc) return rc;
  int64_t p = 0;
  out_off[0] = 0;
  for (size_t i = 0; i < G.e.size(); ++i) {
    for (int32_t v : G.e[i]) out_nodes[p++] = v;
    out_off[i + 1] = p;
  }
  *n_out = (int64_t)G.e.size();
  return 0;
}

// Hyperwedge count and maximum line-graph degree (Algorithm
// "hyperwedge_counting").
int orc_project(int64_t n_edges, const int64_t* off, const int32_t* nodes,
                int64_t* n_wedges, int64_t* max_degree, int64_t* degrees) {
  Hypergraph G;
  if (build(n_edges, off, nodes, G)) return -1;
  LineGraph L = project(G);
  *n_wedges = (int64_t)L.omega.size();
  int64_t mx = 0;
  for (size_t i = 0; i < L.nbr.size(); ++i) {
    mx = std::max<int64_t>(mx, (int64_t)L.nbr[i].size());
    if (degrees) degrees[i] = (int64_t)L.nbr[i].size();
  }
  *max_degree = mx;
  return 0;
}

int orc_count_exact(int64_t n_edges, const int64_t* off, const int32_t* nodes,
                    int32_t theta, int64_t* out_h, int64_t* out_3h) {
  Hypergraph G;
  if (build(n_edges, off, nodes, G)) return -1;
  LineGraph L = project(G);
  exact_count(G, L, theta, nullptr, out_h, out_3h);
  return 0;
}

// Hyperedge profiles (Section 3.1, "Hyperedge Profile (HP)") of every
// hyperedge, from the instances of Algorithm "exact_motif_counting":
// hp_h is |E| x 26, hp_3h is |E| x 431 (row e = hyperedge e after duplicate
// removal); either may be null.
int orc_hyperedge_profile(int64_t n_edges, const int64_t* off, const int32_t* nodes,
                          int32_t theta, int64_t* hp_h, int64_t* hp_3h) {
  Hypergraph G;
  if (build(n_edges, off, nodes, G)) return -1;
  LineGraph L = project(G);
  const int64_t E = (int64_t)G.e.size();
  if (hp_h) std::fill(hp_h, hp_h + E * 26, 0);
  if (hp_3h) std::fill(hp_3h, hp_3h + E * 431, 0);
  int64_t h[26], h3[431];
  exact_count(G, L, theta, nullptr, h, h3, hp_h, hp_3h);
  return 0;
}

// Star node profiles (Section 3.1, "Node Profile (NP)" with the star
// ego-network of "Hypergraph Ego-networks"): the star ego-network of v keeps
// the hyperedges that contain v, E_v, whole; its motif instances are the
// connected triples of E_v (all of them: every pair shares v), classified as
// in G.  np_h is n_nodes x 26, np_3h is n_nodes x 431; either may be null.
int orc_star_node_profile(int64_t n_nodes, int64_t n_edges, const int64_t* off,
                          const int32_t* nodes, int32_t theta, int64_t* np_h,
                          int64_t* np_3h) {
  Hypergraph G;
  if (build(n_edges, off, nodes, G)) return -1;
  if (np_h) std::fill(np_h, np_h + n_nodes * 26, 0);
  if (np_3h) std::fill(np_3h, np_3h + n_nodes * 431, 0);
  auto overlap = [&](int64_t x, int64_t y) {
    int64_t c = 0;
    for (int32_t u : G.e[x]) c += G.eset[y].count(u) ? 1 : 0;
    return c;
  };
  for (const auto& kv : G.ev) {
    const int64_t v = kv.first;
    if (v < 0 || v >= n_nodes) return -1;
    const std::vector<int32_t>& Ev = kv.second;
    for (size_t x = 0; x < Ev.size(); ++x)
      for (size_t y = x + 1; y < Ev.size(); ++y)
        for (size_t z = y + 1; z < Ev.size(); ++z) {
          const int32_t i = Ev[x], j = Ev[y], k = Ev[z];
          auto r = regions(G, i, j, k, overlap(i, j), overlap(j, k), overlap(k, i));
          int h, h3;
          classify(r, theta, &h, &h3);
          if (np_h) np_h[v * 26 + h - 1] += 1;
          if (np_3h) np_3h[v * 431 + h3 - 1] += 1;
        }
  }
  return 0;
}

// MoCHy-E restricted to the outer-loop hyperedges in `anchors`, with the
// hyperedges compared by `rank` (Algorithm "exact_motif_counting" compares
// ids, i < min(j, k); any fixed total order counts every instance exactly
// once, at its centre when open and at its first member when closed).  The
// line-graph rows of the anchors come from the on-the-fly neighbour routine
// (Appendix "on-the-fly", getNeighbors) and the overlaps of neighbour pairs
// from set intersection, so large hypergraphs need not be projected whole.
// With threads > 1 the anchors are shared out among host threads, each with
// its own histogram, summed once at the end (the paper's parallel scheme,
// Section "Parallel and On-the-fly Implementations").
int orc_count_exact_ranked(int64_t n_edges, const int64_t* off, const int32_t* nodes,
                           int32_t theta, const int32_t* anchors, int64_t n_anchors,
                           const int64_t* rank, int32_t threads, int64_t* out_h,
                           int64_t* out_3h) {
  Hypergraph G;
  if (build(n_edges, off, nodes, G)) return -1;
  std::fill(out_h, out_h + 26, 0);
  std::fill(out_3h, out_3h + 431, 0);
  const int64_t E = (int64_t)G.e.size();
  for (int64_t a = 0; a < n_anchors; ++a)
    if (anchors[a] < 0 || anchors[a] >= E) return -1;
  // rank of hyperedge x; the id itself when no order is given
  auto before = [&](int64_t x, int64_t y) {
    return rank ? rank[x] < rank[y] : x < y;
  };
  auto overlap = [&](int64_t x, int64_t y) {
    const auto& s = G.e[x].size() <= G.e[y].size() ? G.e[x] : G.e[y];
    const auto& o = G.e[x].size() <= G.e[y].size() ? G.eset[y] : G.eset[x];
    int64_t c = 0;
    for (int32_t v : s) c += o.count(v) ? 1 : 0;
    return c;
  };
  // the body of the outer loop for one anchor e_i, into h / h3
  auto anchor_body = [&](int32_t i, int64_t* h, int64_t* h3) {
    std::map<int32_t, int32_t> Ni;   // getNeighbors(e_i): e_j -> omega(i, j)
    for (int32_t v : G.e[i])
      for (int32_t j : G.ev.at(v))
        if (j != i) Ni[j] += 1;
    std::vector<std::pair<int32_t, int32_t>> N(Ni.begin(), Ni.end());
    for (size_t x = 0; x < N.size(); ++x)
      for (size_t y = x + 1; y < N.size(); ++y) {
        const int32_t j = N[x].first, k = N[y].first;
        const int64_t wjk = overlap(j, k);
        if (!(wjk == 0 || (before(i, j) && before(i, k)))) continue;
        auto r = regions(G, i, j, k, N[x].second, wjk, N[y].second);
        int hh, t3;
        classify(r, theta, &hh, &t3);
        h[hh - 1] += 1;
        h3[t3 - 1] += 1;
      }
  };
  tables();   // built once, before any thread reads it
  const int nt = threads > 1 ? threads : 1;
  std::vector<std::vector<int64_t>> part(nt, std::vector<int64_t>(26 + 431, 0));
#ifdef _OPENMP
#pragma omp parallel for num_threads(nt) schedule(dynamic, 1)
#endif
  for (int64_t a = 0; a < n_anchors; ++a) {
    int tid = 0;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    anchor_body(anchors[a], part[tid].data(), part[tid].data() + 26);
  }
  for (int t = 0; t < nt; ++t) {
    for (int q = 0; q < 26; ++q) out_h[q] += part[t][q];
    for (int q = 0; q < 431; ++q) out_3h[q] += part[t][26 + q];
  }
  return 0;
}

// MoCHy-E restricted to the outer-loop hyperedges in `anchors` (ids
// compared as in Algorithm "exact_motif_counting"), one thread.
int orc_count_exact_subset(int64_t n_edges, const int64_t* off,
                           const int32_t* nodes, int32_t theta,
                           const int32_t* anchors, int64_t n_anchors,
                           int64_t* out_h, int64_t* out_3h) {
  return orc_count_exact_ranked(n_edges, off, nodes, theta, anchors, n_anchors, nullptr, 1,
                                out_h, out_3h);
}

// Line-graph degree |N_{e_i}| of every hyperedge (Section 2.1 "Line Graph":
// the hyperedges other than e_i that share a node with it), from the
// incidence lists: |(union of E_v over v in e_i) \ {e_i}|, each hyperedge
// counted once by marking it with the current i.
int orc_line_degrees(int64_t n_edges, const int64_t* off, const int32_t* nodes,
                     int32_t threads, int64_t* degrees) {
  Hypergraph G;
  if (build(n_edges, off, nodes, G)) return -1;
  const int64_t E = (int64_t)G.e.size();
  const int nt = threads > 1 ? threads : 1;
#ifdef _OPENMP
#pragma omp parallel num_threads(nt)
#endif
  {
    std::vector<int64_t> mark(E, -1);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 64)
#endif
    for (int64_t i = 0; i < E; ++i) {
      int64_t d = 0;
      mark[i] = i;
      for (int32_t v : G.e[i])
        for (int32_t j : G.ev.at(v))
          if (mark[j] != i) {
            mark[j] = i;
            ++d;
          }
      degrees[i] = d;
    }
  }
  return 0;
}

// method 1 = MoCHy-A (samples = s), 2 = MoCHy-A+ (samples = r).
int orc_count_sampled(int64_t n_edges, const int64_t* off, const int32_t* nodes,
                      int32_t theta, int method, int64_t samples, uint64_t seed,
                      int64_t* raw_h, int64_t* raw_3h, double* est_h,
                      double* est_3h) {
  Hypergraph G;
  if (build(n_edges, off, nodes, G)) return -1;
  if (samples <= 0) return -1;
  LineGraph L = project(G);
  std::fill(raw_h, raw_h + 26, 0);
  std::fill(raw_3h, raw_3h + 431, 0);
  const Tables& T = tables();
  if (method == 1) {
    if (G.e.empty()) return -1;
    count_A(G, L, theta, samples, seed, raw_h, raw_3h);
    // Algorithm "sampling_ver1": rescale by |E| / (3 s)
    for (int t = 0; t < 26; ++t)
      est_h[t] = (double)raw_h[t] * (double)G.e.size() / (3.0 * (double)samples);
    for (int t = 0; t < 431; ++t)
      est_3h[t] = (double)raw_3h[t] * (double)G.e.size() / (3.0 * (double)samples);
  } else if (method == 2) {
    if (L.omega.empty()) return -1;
    count_Aplus(G, L, theta, samples, seed, raw_h, raw_3h);
    // Eq. "mht:scale": rescale by |wedges| / (w[t] r), w = 2 open, 3 closed
    const double nw = (double)L.omega.size();
    for (int t = 0; t < 26; ++t) {
      const double w = T.h_open[t] ? 2.0 : 3.0;
      est_h[t] = (double)raw_h[t] * nw / (w * (double)samples);
    }
    for (int t = 0; t < 431; ++t) {
      const double w = T.h_open[T.t_to_h[t] - 1] ? 2.0 : 3.0;
      est_3h[t] = (double)raw_3h[t] * nw / (w * (double)samples);
    }
  } else {
    return -1;
  }
  return 0;
}

// The body of MoCHy-A run once for every hyperedge (method 1) or the body of
// MoCHy-A+ run once for every hyperwedge (method 2), without sampling.  By
// Eq. "mbt" / Eq. "mht" these must give 3 M[t] and w[t] M[t] exactly.
int orc_count_all_anchors(int64_t n_edges, const int64_t* off,
                          const int32_t* nodes, int32_t theta, int method,
                          int64_t* raw_h, int64_t* raw_3h) {
  Hypergraph G;
  if (build(n_edges, off, nodes, G)) return -1;
  LineGraph L = project(G);
  std::fill(raw_h, raw_h + 26, 0);
  std::fill(raw_3h, raw_3h + 431, 0);
  if (method == 1) {
    for (int64_t i = 0; i < (int64_t)G.e.size(); ++i) {
      const auto& Ni = L.nbr[i];
      std::unordered_set<int32_t> inNi(Ni.begin(), Ni.end());
      for (int32_t j : Ni) {
        std::set<int32_t> cand(Ni.begin(), Ni.end());
        cand.insert(L.nbr[j].begin(), L.nbr[j].end());
        cand.erase((int32_t)i);
        cand.erase(j);
        for (int32_t k : cand)
          if (!inNi.count(k) || j < k) add_instance(G, L, theta, i, j, k, raw_h, raw_3h);
      }
    }
  } else if (method == 2) {
    for (auto& w : sorted_wedges(L)) {
      std::set<int32_t> cand(L.nbr[w.first].begin(), L.nbr[w.first].end());
      cand.insert(L.nbr[w.second].begin(), L.nbr[w.second].end());
      cand.erase(w.first);
      cand.erase(w.second);
      for (int32_t k : cand) add_instance(G, L, theta, w.first, w.second, k, raw_h, raw_3h);
    }
  } else {
    return -1;
  }
  return 0;
}

// One randomized copy; out_off must hold n_edges+1 entries and out_nodes
// sum |e| entries (a copy never has more).
int orc_randomize(int64_t n_nodes, int64_t n_edges, const int64_t* off,
                  const int32_t* nodes, uint64_t seed, uint32_t copy,
                  int64_t* out_off, int32_t* out_nodes, int64_t* n_out) {
  Hypergraph G;
  if (build(n_edges, off, nodes, G)) return -1;
  for (auto& e : G.e)
    if (e.back() >= n_nodes) return -1;
  std::vector<std::vector<int32_t>> R;
  randomize(G, n_nodes, seed, copy, R);
  int64_t p = 0;
  out_off[0] = 0;
  for (size_t i = 0; i < R.size(); ++i) {
    for (int32_t v : R[i]) out_nodes[p++] = v;
    out_off[i + 1] = p;
  }
  *n_out = (int64_t)R.size();
  return 0;
}

// Significance and CP of the input against n_random copies.
int orc_profile(int64_t n_nodes, int64_t n_edges, const int64_t* off,
                const int32_t* nodes, int32_t theta, int32_t n_random,
                uint64_t seed, double eps, double* sig_h, double* cp_h,
                double* sig_3h, double* cp_3h, int64_t* counts_h,
                int64_t* counts_3h, int32_t* degenerate) {
  if (n_random <= 0) return -1;
  Hypergraph G;
  if (build(n_edges, off, nodes, G)) return -1;
  // counts_h / counts_3h receive (1 + n_random) rows: the input, then copies
  {
    LineGraph L = project(G);
    exact_count(G, L, theta, nullptr, counts_h, counts_3h);
  }
  std::vector<int64_t> sum_h(26, 0), sum_3h(431, 0);
  for (int32_t c = 0; c < n_random; ++c) {
    std::vector<std::vector<int32_t>> R;
    randomize(G, n_nodes, seed, (uint32_t)c, R);
    Hypergraph H;
    H.e = R;
    for (size_t i = 0; i < H.e.size(); ++i) {
      H.eset.emplace_back(H.e[i].begin(), H.e[i].end());
      for (int32_t v : H.e[i]) H.ev[v].push_back((int32_t)i);
    }
    LineGraph L = project(H);
    int64_t* ch = counts_h + 26 * (1 + c);
    int64_t* c3 = counts_3h + 431 * (1 + c);
    exact_count(H, L, theta, nullptr, ch, c3);
    for (int t = 0; t < 26; ++t) sum_h[t] += ch[t];
    for (int t = 0; t < 431; ++t) sum_3h[t] += c3[t];
  }
  std::vector<double> mr_h(26), mr_3h(431);
  for (int t = 0; t < 26; ++t) mr_h[t] = (double)sum_h[t] / (double)n_random;
  for (int t = 0; t < 431; ++t) mr_3h[t] = (double)sum_3h[t] / (double)n_random;
  int d1 = 0, d2 = 0;
  significance_cp(counts_h, mr_h.data(), 26, eps, sig_h, cp_h, &d1);
  significance_cp(counts_3h, mr_3h.data(), 431, eps, sig_3h, cp_3h, &d2);
  degenerate[0] = d1;
  degenerate[1] = d2;
  return 0;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Extensions: kh-motifs, radial node profiles, instance enumeration, the
// significance and CP on their own.
// ---------------------------------------------------------------------------
extern "C" {

// kh-motif tables for k states (Section 4.1 "Extensions Beyond Ternary";
// their number is X(k) of Appendix "Number of kH-motifs"): lut has k^7
// entries (code = sum_p state_p k^p -> id, 0 = no motif); pattern (n x 7)
// and to_h (n) are filled for the n motifs when non-null and n <= cap.
int64_t orc_kh_tables(int k, int32_t* lut, uint8_t* pattern, int32_t* to_h, int64_t cap) {
  if (k < 2 || k > 6) return -1;
  const KTables& K = k_tables(k);
  const int64_t n = (int64_t)K.pattern.size();
  if (lut) std::memcpy(lut, K.lut.data(), K.lut.size() * sizeof(int32_t));
  if (n <= cap) {
    for (int64_t i = 0; i < n; ++i) {
      if (pattern)
        for (int r = 0; r < 7; ++r) pattern[i * 7 + r] = (uint8_t)K.pattern[i][r];
      if (to_h) to_h[i] = K.to_h[i];
    }
  }
  return n;
}

// Exact kh-motif counts: Algorithm "exact_motif_counting" with h(.) replaced
// by the k-state classification of the seven regions (Section 4.1; the
// regions from Lemma "motif:time").  thr holds the k - 2 ascending
// thresholds; out_kh has X(k) entries, out_h 26.
int orc_count_exact_kh(int64_t n_edges, const int64_t* off, const int32_t* nodes, int32_t k,
                       const int32_t* thr, int64_t* out_h, int64_t* out_kh) {
  if (k < 2 || k > 6) return -1;
  for (int m = 0; m + 1 < k - 2; ++m)
    if (thr[m] < 1 || thr[m + 1] <= thr[m]) return -1;
  if (k > 2 && thr[0] < 1) return -1;
  Hypergraph G;
  if (build(n_edges, off, nodes, G)) return -1;
  LineGraph L = project(G);
  const KTables& K = k_tables(k);
  std::fill(out_h, out_h + 26, 0);
  std::fill(out_kh, out_kh + K.pattern.size(), 0);
  const int64_t E = (int64_t)G.e.size();
  for (int64_t i = 0; i < E; ++i) {
    const auto& N = L.nbr[i];
    for (size_t x = 0; x < N.size(); ++x)
      for (size_t y = x + 1; y < N.size(); ++y) {
        const int32_t j = N[x], kk = N[y];
        const int32_t wjk = omega_of(L, j, kk);
        if (!(wjk == 0 || i < std::min(j, kk))) continue;
        auto r = regions(G, i, j, kk, omega_of(L, i, j), wjk, omega_of(L, kk, i));
        int64_t code = 0, pw = 1;
        for (int p = 0; p < 7; ++p) {
          code += k_state(r[p], k, thr) * pw;
          pw *= k;
        }
        const int id = K.lut[(size_t)code];
        if (id <= 0) return -2;
        out_kh[id - 1] += 1;
        out_h[K.to_h[id - 1] - 1] += 1;
      }
  }
  return 0;
}

// Radial node profiles (Section 3.1, "Node Profile (NP)" with the radial
// ego-network of "Hypergraph Ego-networks"): V_v is the union of the
// hyperedges that contain v, R_v the hyperedges that are subsets of V_v; the
// radial ego-network of v is (V_v, R_v) and its instances are the connected
// triples of R_v, counted here by MoCHy-E on that subhypergraph.  Hyperedges
// are kept whole, so regions and motifs are those in G.  np_h is n_nodes x
// 26, np_3h n_nodes x 431; either may be null.
int orc_radial_node_profile(int64_t n_nodes, int64_t n_edges, const int64_t* off,
                            const int32_t* nodes, int32_t theta, int64_t* np_h,
                            int64_t* np_3h) {
  Hypergraph G;
  if (build(n_edges, off, nodes, G)) return -1;
  if (np_h) std::fill(np_h, np_h + n_nodes * 26, 0);
  if (np_3h) std::fill(np_3h, np_3h + n_nodes * 431, 0);
  for (const auto& kv : G.ev) {
    const int64_t v = kv.first;
    if (v < 0 || v >= n_nodes) return -1;
    std::unordered_set<int32_t> Vv;
    for (int32_t e : kv.second) Vv.insert(G.e[e].begin(), G.e[e].end());
    Hypergraph R;   // (V_v, R_v), hyperedges in the order of G
    for (size_t i = 0; i < G.e.size(); ++i) {
      bool inside = true;
      for (int32_t u : G.e[i]) inside = inside && Vv.count(u) > 0;
      if (inside) R.e.push_back(G.e[i]);
    }
    for (size_t i = 0; i < R.e.size(); ++i) {
      R.eset.emplace_back(R.e[i].begin(), R.e[i].end());
      for (int32_t u : R.e[i]) R.ev[u].push_back((int32_t)i);
    }
    LineGraph L = project(R);
    int64_t h[26], h3[431];
    exact_count(R, L, theta, nullptr, h, h3);
    for (int t = 0; t < 26; ++t)
      if (np_h) np_h[v * 26 + t] = h[t];
    for (int t = 0; t < 431; ++t)
      if (np_3h) np_3h[v * 431 + t] = h3[t];
  }
  return 0;
}

// Algorithm "alg:enum" (MoCHy-E_ENUM): every instance written once with its
// motifs, as (i, j, k, h, 3h) with the three ids ascending (ids after
// duplicate removal); *n_out receives the number of instances, of which the
// first min(n, cap) are written to out (cap x 5) in the order the algorithm
// meets them.
int orc_enumerate(int64_t n_edges, const int64_t* off, const int32_t* nodes, int32_t theta,
                  int64_t cap, int32_t* out, int64_t* n_out) {
  Hypergraph G;
  if (build(n_edges, off, nodes, G)) return -1;
  LineGraph L = project(G);
  const int64_t E = (int64_t)G.e.size();
  int64_t n = 0;
  for (int64_t i = 0; i < E; ++i) {
    const auto& N = L.nbr[i];
    for (size_t x = 0; x < N.size(); ++x)
      for (size_t y = x + 1; y < N.size(); ++y) {
        const int32_t j = N[x], k = N[y];
        const int32_t wjk = omega_of(L, j, k);
        if (!(wjk == 0 || i < std::min(j, k))) continue;
        auto r = regions(G, i, j, k, omega_of(L, i, j), wjk, omega_of(L, k, i));
        int h, h3;
        classify(r, theta, &h, &h3);
        if (n < cap) {
          int32_t ids[3] = {(int32_t)i, j, k};
          std::sort(ids, ids + 3);
          int32_t* o = out + n * 5;
          o[0] = ids[0];
          o[1] = ids[1];
          o[2] = ids[2];
          o[3] = h;
          o[4] = h3;
        }
        ++n;
      }
  }
  *n_out = n;
  return 0;
}

// Eq. "significance" and Eq. "cp" for n motifs: M are the input's counts,
// sum_rand the counts summed over n_random randomized copies (M_rand is
// their mean, reading R9).
int orc_significance_cp(const int64_t* M, const int64_t* sum_rand, int32_t n_random, int32_t n,
                        double eps, double* sig, double* cp, int32_t* degenerate) {
  if (n_random <= 0 || n <= 0) return -1;
  std::vector<double> mr(n);
  for (int t = 0; t < n; ++t) mr[t] = (double)sum_rand[t] / (double)n_random;
  int d = 0;
  significance_cp(M, mr.data(), n, eps, sig, cp, &d);
  *degenerate = d;
  return 0;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// MoCHy-A+ without the line graph (Section 3.4 "Motif Counting without Line
// Graphs"; Appendix "Details of On-the-Fly MoCHy", Algorithms "alg_memdeg"
// (basic) and "alg_memdeg_adv" (advanced)).
//
// Readings: (R13) a uniformly random hyperwedge is drawn exactly as by
// MoCHy-A+ (readings R6, R7: index floor(u |wedges| / 2^64) in ascending
// (i, j) order), so that the on-the-fly runs classify the same hyperwedges
// as the projected one; the number of neighbours after each hyperedge, which
// that order needs, comes from the same pass as the degrees d_i.  (R14) the
// budget b counts memoized neighbour entries (sum of d_l over memoized
// hyperedges).  (R15) when even an empty memo cannot hold N_{e_l}
// (d_l > b), N_{e_l} is computed for the current hyperwedge only and not
// memoized (the eviction loop of the algorithms would not end).
// ---------------------------------------------------------------------------
namespace {

// getNeighbors(e, G): hyperedge -> omega over the incidence lists
std::map<int32_t, int32_t> get_neighbors(const Hypergraph& G, int32_t e) {
  std::map<int32_t, int32_t> n;
  for (int32_t v : G.e[e])
    for (int32_t f : G.ev.at(v))
      if (f != e) n[f] += 1;
  return n;
}

struct OnTheFlyStats {
  int64_t built = 0;     // getNeighbors calls
  int64_t evicted = 0;   // neighbourhoods evicted to make room
};

// The memo A with capacity cap and the priority queue Q of memoized
// hyperedges, lowest degree popped first (Appendix "on-the-fly": Q
// prioritizes high-degree hyperedges, so a low-degree one is evicted).
struct Memo {
  const Hypergraph& G;
  const std::vector<int64_t>& d;
  int64_t cap;
  std::map<int32_t, std::map<int32_t, int32_t>> A;
  std::set<std::pair<int64_t, int32_t>> Q;
  OnTheFlyStats st;
  Memo(const Hypergraph& g, const std::vector<int64_t>& deg, int64_t b) : G(g), d(deg), cap(b) {}

  bool in_q(int32_t l) const { return Q.count({d[l], l}) > 0; }

  // the body of the "for each l in {i, j}" memo loop for one l; returns
  // N_{e_l} (memoized, or computed for this use only, reading R15)
  const std::map<int32_t, int32_t>& fetch(int32_t l, int32_t i, int32_t j,
                                          std::map<int32_t, int32_t>& scratch) {
    auto it = A.find(l);
    if (it != A.end()) return it->second;
    std::vector<std::pair<int64_t, int32_t>> held;   // popped i or j, pushed back below
    while (cap < d[l] && !Q.empty()) {
      auto m = *Q.begin();
      Q.erase(Q.begin());
      if (m.second != i && m.second != j) {
        cap += d[m.second];
        A.erase(m.second);
        ++st.evicted;
      } else {
        held.push_back(m);
      }
    }
    for (auto& h : held) Q.insert(h);
    ++st.built;
    if (cap < d[l]) {
      scratch = get_neighbors(G, l);
      return scratch;
    }
    A[l] = get_neighbors(G, l);
    cap -= d[l];
    Q.insert({d[l], l});
    return A[l];
  }

  void drop(int32_t l) {   // Algorithm alg_memdeg_adv: a key's group is done
    auto it = A.find(l);
    if (it == A.end()) return;
    Q.erase({d[l], l});
    cap += d[l];
    A.erase(it);
  }
};

// The classification of every e_k in N_i u N_j \ {e_i, e_j} (the counting
// loop shared by both algorithms and by Algorithm "sampling_ver2").
void count_union(const Hypergraph& G, int32_t theta, int32_t i, int32_t j,
                 const std::map<int32_t, int32_t>& Ni, const std::map<int32_t, int32_t>& Nj,
                 int64_t* raw_h, int64_t* raw_3h) {
  const int64_t wij = Ni.count(j) ? Ni.at(j) : 0;
  std::set<int32_t> cand;
  for (auto& kv : Ni) cand.insert(kv.first);
  for (auto& kv : Nj) cand.insert(kv.first);
  cand.erase(i);
  cand.erase(j);
  for (int32_t k : cand) {
    auto a = Ni.find(k);
    auto b = Nj.find(k);
    const int64_t wik = a == Ni.end() ? 0 : a->second;
    const int64_t wjk = b == Nj.end() ? 0 : b->second;
    auto r = regions(G, i, j, k, wij, wjk, wik);
    int h, h3;
    classify(r, theta, &h, &h3);
    raw_h[h - 1] += 1;
    raw_3h[h3 - 1] += 1;
  }
}

}  // namespace

extern "C" {

// method 1 = basic (Algorithm "alg_memdeg"), 2 = advanced
// (Algorithm "alg_memdeg_adv"); budget = b in neighbour entries.  Estimates
// as Algorithm "sampling_ver2" (open w = 2, closed w = 3).  stats (may be
// null): getNeighbors calls, evictions.
int orc_count_aplus_onthefly(int64_t n_edges, const int64_t* off, const int32_t* nodes,
                             int32_t theta, int method, int64_t samples, uint64_t seed,
                             int64_t budget, int64_t* raw_h, int64_t* raw_3h, double* est_h,
                             double* est_3h, int64_t* stats) {
  Hypergraph G;
  if (build(n_edges, off, nodes, G)) return -1;
  if (samples <= 0 || budget < 0 || (method != 1 && method != 2)) return -1;
  const int64_t E = (int64_t)G.e.size();
  // the degrees d_i in the line graph, and the neighbours after each i
  std::vector<int64_t> d(E, 0), up(E, 0);
  for (int64_t i = 0; i < E; ++i) {
    auto n = get_neighbors(G, (int32_t)i);
    d[i] = (int64_t)n.size();
    for (auto& kv : n) up[i] += kv.first > i ? 1 : 0;
  }
  std::vector<int64_t> upre(E + 1, 0);
  for (int64_t i = 0; i < E; ++i) upre[i + 1] = upre[i] + up[i];
  const uint64_t nw = (uint64_t)upre[E];
  if (nw == 0) return -1;
  // the n-th sampled hyperwedge (reading R13)
  auto sample = [&](int64_t n, Memo& memo, std::map<int32_t, int32_t>& scratch) {
    const int64_t w = (int64_t)scale_index(draw_u64(seed, (uint64_t)n, kStreamWedgeSample, 0), nw);
    const int64_t i = (int64_t)(std::upper_bound(upre.begin(), upre.end(), w) - upre.begin()) - 1;
    const auto& Ni = memo.fetch((int32_t)i, (int32_t)i, -1, scratch);
    int64_t o = w - upre[i];
    int32_t j = -1;
    for (auto& kv : Ni)
      if (kv.first > i && o-- == 0) { j = kv.first; break; }
    return std::make_pair((int32_t)i, j);
  };
  std::fill(raw_h, raw_h + 26, 0);
  std::fill(raw_3h, raw_3h + 431, 0);
  Memo memo(G, d, budget);
  std::map<int32_t, int32_t> si, sj;
  if (method == 1) {
    for (int64_t n = 0; n < samples; ++n) {
      auto ij = sample(n, memo, si);
      const int32_t i = ij.first, j = ij.second;
      // for each l in {i, j}: memoized or fetched (Algorithm alg_memdeg)
      std::map<int32_t, int32_t> Ni = memo.fetch(i, i, j, si);
      const auto& Nj = memo.fetch(j, i, j, sj);
      for (int32_t l : {i, j})
        if (memo.A.count(l) && !memo.in_q(l)) memo.Q.insert({d[l], l});
      count_union(G, theta, i, j, Ni, Nj, raw_h, raw_3h);
    }
  } else {
    // collect the r hyperwedges, grouped by their key hyperedge (the one of
    // larger (d, id)), then processed in descending (d, id) of the keys
    std::map<std::pair<int64_t, int32_t>, std::vector<std::pair<int32_t, int32_t>>,
             std::greater<std::pair<int64_t, int32_t>>> W;
    // (a draw reads N_{e_i} through the same memo, reading R13)
    for (int64_t n = 0; n < samples; ++n) {
      auto ij = sample(n, memo, si);
      const int32_t i = ij.first, j = ij.second;
      const bool i_key = d[i] > d[j] || (d[i] == d[j] && i > j);
      const int32_t key = i_key ? i : j;
      W[{d[key], key}].push_back(ij);
    }
    for (auto& grp : W) {
      const int32_t key = grp.first.second;
      for (auto& ij : grp.second) {
        const int32_t i = ij.first, j = ij.second;
        std::map<int32_t, int32_t> Ni = memo.fetch(i, i, j, si);
        const auto& Nj = memo.fetch(j, i, j, sj);
        count_union(G, theta, i, j, Ni, Nj, raw_h, raw_3h);
      }
      memo.drop(key);
    }
  }
  const Tables& T = tables();
  for (int t = 0; t < 26; ++t) {
    const double w = T.h_open[t] ? 2.0 : 3.0;
    est_h[t] = (double)raw_h[t] * (double)nw / (w * (double)samples);
  }
  for (int t = 0; t < 431; ++t) {
    const double w = T.h_open[T.t_to_h[t] - 1] ? 2.0 : 3.0;
    est_3h[t] = (double)raw_3h[t] * (double)nw / (w * (double)samples);
  }
  if (stats) {
    stats[0] = memo.st.built;
    stats[1] = memo.st.evicted;
    stats[2] = (int64_t)nw;
  }
  return 0;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Per-row shares of the exact count when open instances are counted per
// centre from all pairs of its neighbours (the decomposition the library's
// split count uses; not one of the paper's algorithms, but an identity
// between its counts).
//
// For a centre e_c and neighbours e_p, e_q with omega(c,p) + omega(c,q) <=
// |e_c|, "as if open" classifies {c; p, q} with the regions of an open
// instance centred at c (Lemma "motif:time" with omega(p,q) = 0 and no
// triple intersection).  An open instance is met exactly so at its centre
// and nowhere else; a closed instance is met so at each of its three
// centres where the condition holds.  Hence the exact count (Algorithm
// "exact_motif_counting") equals the sum over rows r of
//   (every pair of neighbours of r, as if open at r)
// + (for each closed instance whose first member in `rank` is r: its motif,
//    minus its "as if open" term at each of its three centres),
// which is what the share of a row is.  Shares may be negative.
// ---------------------------------------------------------------------------
extern "C" {

int orc_count_split_rows(int64_t n_edges, const int64_t* off, const int32_t* nodes,
                         int32_t theta, const int32_t* rows, int64_t n_rows, const int64_t* rank,
                         int32_t threads, int64_t* out_h, int64_t* out_3h) {
  Hypergraph G;
  if (build(n_edges, off, nodes, G)) return -1;
  std::fill(out_h, out_h + 26, 0);
  std::fill(out_3h, out_3h + 431, 0);
  const int64_t E = (int64_t)G.e.size();
  for (int64_t a = 0; a < n_rows; ++a)
    if (rows[a] < 0 || rows[a] >= E) return -1;
  auto before = [&](int64_t x, int64_t y) { return rank ? rank[x] < rank[y] : x < y; };
  auto overlap = [&](int64_t x, int64_t y) {
    const auto& s = G.e[x].size() <= G.e[y].size() ? G.e[x] : G.e[y];
    const auto& o = G.e[x].size() <= G.e[y].size() ? G.eset[y] : G.eset[x];
    int64_t c = 0;
    for (int32_t v : s) c += o.count(v) ? 1 : 0;
    return c;
  };
  // add (sign +1 / -1) the "as if open" term of centre c with leaves p, q
  auto as_if_open = [&](int64_t c, int64_t p, int64_t q, int64_t wcp, int64_t wcq, int64_t sign,
                        int64_t* h, int64_t* h3) {
    const int64_t A = (int64_t)G.e[c].size();
    if (wcp + wcq > A) return;
    const std::array<int64_t, 7> r = {A - wcp - wcq, (int64_t)G.e[p].size() - wcp,
                                      (int64_t)G.e[q].size() - wcq, wcp, 0, wcq, 0};
    int hh, t3;
    classify(r, theta, &hh, &t3);
    h[hh - 1] += sign;
    h3[t3 - 1] += sign;
  };
  auto row_body = [&](int32_t r, int64_t* h, int64_t* h3) {
    const auto Nr = get_neighbors(G, r);
    std::vector<std::pair<int32_t, int32_t>> N(Nr.begin(), Nr.end());
    for (size_t x = 0; x < N.size(); ++x)
      for (size_t y = x + 1; y < N.size(); ++y) {
        const int32_t j = N[x].first, k = N[y].first;
        const int64_t wrj = N[x].second, wrk = N[y].second;
        as_if_open(r, j, k, wrj, wrk, +1, h, h3);
        const int64_t wjk = overlap(j, k);
        if (wjk == 0 || !(before(r, j) && before(r, k))) continue;
        auto reg = regions(G, r, j, k, wrj, wjk, wrk);
        int hh, t3;
        classify(reg, theta, &hh, &t3);
        h[hh - 1] += 1;
        h3[t3 - 1] += 1;
        as_if_open(r, j, k, wrj, wrk, -1, h, h3);
        as_if_open(j, r, k, wrj, wjk, -1, h, h3);
        as_if_open(k, r, j, wrk, wjk, -1, h, h3);
      }
  };
  tables();
  const int nt = threads > 1 ? threads : 1;
  std::vector<std::vector<int64_t>> part(nt, std::vector<int64_t>(26 + 431, 0));
#ifdef _OPENMP
#pragma omp parallel for num_threads(nt) schedule(dynamic, 1)
#endif
  for (int64_t a = 0; a < n_rows; ++a) {
    int tid = 0;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    row_body(rows[a], part[tid].data(), part[tid].data() + 26);
  }
  for (int t = 0; t < nt; ++t) {
    for (int q = 0; q < 26; ++q) out_h[q] += part[t][q];
    for (int q = 0; q < 431; ++q) out_3h[q] += part[t][26 + q];
  }
  return 0;
}

}  // extern "C"
