// Host setup, once per topology: triplet stream -> the CSR pattern that two
// transposes of it give (Section 4.2, Table "build pattern"; built per node
// on the host's cores, bit-identical to the transposes), the map C and its inverse,
// projective constraints folded into the pattern (Section 5.1), consistent
// mass, element rest data, nested-dissection ordering of the free nodes and
// the multifrontal symbolic analysis + level schedule (Section 6.1,
// Eq. "regional problem").  Plain C++; no CUDA.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <new>
#include <numeric>
#include <thread>

#include "fe_ctx.h"

namespace fe {

int set_error(const fe_ctx *c, int code, const std::string &msg) {
  if (c) const_cast<fe_ctx *>(c)->err = msg;
  return code;
}

namespace {

inline double det3(const double *m) {  // row-major 3x3
  return m[0] * (m[4] * m[8] - m[5] * m[7]) - m[1] * (m[3] * m[8] - m[5] * m[6]) +
         m[2] * (m[3] * m[7] - m[4] * m[6]);
}

inline void inv3(const double *m, double *o) {  // row-major 3x3 inverse
  double d = det3(m);
  o[0] = (m[4] * m[8] - m[5] * m[7]) / d;
  o[1] = (m[2] * m[7] - m[1] * m[8]) / d;
  o[2] = (m[1] * m[5] - m[2] * m[4]) / d;
  o[3] = (m[5] * m[6] - m[3] * m[8]) / d;
  o[4] = (m[0] * m[8] - m[2] * m[6]) / d;
  o[5] = (m[2] * m[3] - m[0] * m[5]) / d;
  o[6] = (m[3] * m[7] - m[4] * m[6]) / d;
  o[7] = (m[1] * m[6] - m[0] * m[7]) / d;
  o[8] = (m[0] * m[4] - m[1] * m[3]) / d;
}

// Trilinear shape-function derivatives dN[a][r] at xi (corner order a = dx+2dy+4dz).
void hex_dshape(const double xi[3], double N[8], double dN[8][3]) {
  for (int a = 0; a < 8; ++a) {
    double c[3] = {double(2 * (a & 1) - 1), double(2 * ((a >> 1) & 1) - 1),
                   double(2 * ((a >> 2) & 1) - 1)};
    double f[3] = {1 + c[0] * xi[0], 1 + c[1] * xi[1], 1 + c[2] * xi[2]};
    N[a] = f[0] * f[1] * f[2] / 8.0;
    dN[a][0] = c[0] * f[1] * f[2] / 8.0;
    dN[a][1] = c[1] * f[0] * f[2] / 8.0;
    dN[a][2] = c[2] * f[0] * f[1] / 8.0;
  }
}

void hex_gauss(int q, double xi[3]) {
  const double g = 1.0 / std::sqrt(3.0);
  xi[0] = (2 * (q & 1) - 1) * g;
  xi[1] = (2 * ((q >> 1) & 1) - 1) * g;
  xi[2] = (2 * ((q >> 2) & 1) - 1) * g;
}

// Host threads for the setup: the hardware's, capped by FE_HOST_THREADS
// when that is set to a positive integer, and by 64.
unsigned host_threads() {
  unsigned nt = std::thread::hardware_concurrency();
  if (const char *env = std::getenv("FE_HOST_THREADS")) {
    const long v = std::strtol(env, nullptr, 10);
    if (v > 0) nt = unsigned(std::min<long>(v, 64));
  }
  return std::max(1u, std::min(nt, 64u));
}

// Runs f(begin, end) over [0, count) in chunks on the host's cores.  Each
// index's output must go to a position fixed beforehand, so the result does
// not depend on the number of threads or on their order.
template <class F>
void parallel_chunks(int64_t count, int64_t chunk, F &&f) {
  const unsigned nt = host_threads();
  if (count <= chunk || nt == 1) {
    if (count > 0) f(int64_t(0), count);
    return;
  }
  std::atomic<int64_t> next{0};
  std::atomic<bool> failed{false};
  auto work = [&] {
    try {
      for (;;) {
        const int64_t b = next.fetch_add(chunk);
        if (b >= count || failed.load()) break;
        f(b, std::min(count, b + chunk));
      }
    } catch (...) {  // an exception must not leave a worker thread
      failed.store(true);
    }
  };
  std::vector<std::thread> pool;
  for (unsigned i = 1; i < nt; ++i) {
    try {
      pool.emplace_back(work);
    } catch (...) {
      break;  // fewer threads: the calling thread still takes every chunk left
    }
  }
  work();
  for (auto &t : pool) t.join();
  if (failed.load()) throw std::bad_alloc();  // the only exception the bodies raise
}

// ------------------------------------------------------------------ pattern
// The CSR pattern of the projected matrix, C and its inverse, as the two
// transposes of the uncompressed triplet structure define them (rows
// ascending, columns ascending, equal (row, col) merged with their triplets in
// fill order), built row by row: a node's rows collect the (column, triplet)
// pairs of the elements around the node, sorted by column and then triplet id.
// Counts fix every row's output range first, so the nodes build in parallel.
// All rows of a node carry the same columns; a fixed row keeps a lone
// diagonal slot, a fixed column is dropped (C = -1).
int build_csr(fe_ctx *c) {
  const int npe = c->npe;
  const int64_t E = c->n_elems, n = c->n, nn = c->n_nodes;
  const int64_t bpe = int64_t(npe) * npe * 9;  // triplets per element
  c->ntrip = E * bpe;
  if (c->ntrip >= (int64_t(1) << 31)) return set_error(c, FE_ERR_ARG, "too many triplets for int32 ids");
  const int32_t *conn = c->conn.data();
  const int8_t *fx = c->fixed_dof.data();
  // node incidence lists (element-major, ascending); the force gather uses them too
  c->node_ptr.assign(nn + 1, 0);
  for (int64_t k = 0; k < E * npe; ++k) c->node_ptr[conn[k] + 1]++;
  for (int64_t i = 0; i < nn; ++i) c->node_ptr[i + 1] += c->node_ptr[i];
  c->node_src.assign(E * npe, 0);
  {
    std::vector<int32_t> next(c->node_ptr.begin(), c->node_ptr.end() - 1);
    for (int64_t k = 0; k < E * npe; ++k) c->node_src[next[conn[k]]++] = int32_t(k);
  }
  // free DOFs per element = kept columns of each of its free rows
  std::vector<int32_t> kept_e(E);
  for (int64_t e = 0; e < E; ++e) {
    int32_t k = 0;
    for (int a = 0; a < npe; ++a)
      for (int j = 0; j < 3; ++j) k += fx[3 * int64_t(conn[e * npe + a]) + j] ? 0 : 1;
    kept_e[e] = k;
  }
  for (int64_t v = 0; v < nn; ++v)
    if (c->node_ptr[v] == c->node_ptr[v + 1] && !(fx[3 * v] && fx[3 * v + 1] && fx[3 * v + 2]))
      return set_error(c, FE_ERR_ARG, "node " + std::to_string(v) + " is free but belongs to no element");
  std::vector<int64_t> rp(n + 1, 0);  // kept triplets per row
  for (int64_t v = 0; v < nn; ++v) {
    int64_t cnt = 0;
    for (int32_t p = c->node_ptr[v]; p < c->node_ptr[v + 1]; ++p) cnt += kept_e[c->node_src[p] / npe];
    for (int i = 0; i < 3; ++i) rp[3 * v + i + 1] = fx[3 * v + i] ? 0 : cnt;
  }
  for (int64_t i = 0; i < n; ++i) rp[i + 1] += rp[i];
  const int64_t kept = rp[n];
  c->slot_src.assign(kept, 0);
  std::vector<int32_t> x_col(kept);
  std::vector<int32_t> uniq(nn, 0);  // distinct columns of a node's free rows
  const int32_t *nptr = c->node_ptr.data(), *nsrc = c->node_src.data();
  int32_t *ssrc = c->slot_src.data();
  parallel_chunks(nn, 512, [&](int64_t v0, int64_t v1) {
    std::vector<uint64_t> keys;  // column << 32 | triplet id of the node's row 0
    for (int64_t v = v0; v < v1; ++v) {
      if (fx[3 * v] && fx[3 * v + 1] && fx[3 * v + 2]) continue;
      keys.clear();
      for (int32_t p = nptr[v]; p < nptr[v + 1]; ++p) {
        const int64_t e = nsrc[p] / npe, a = nsrc[p] % npe;
        const int64_t tb = (e * npe + a) * npe * 9;
        for (int bb = 0; bb < npe; ++bb) {
          const int64_t w = conn[e * npe + bb];
          for (int k = 0; k < 3; ++k)
            if (!fx[3 * w + k]) keys.push_back(uint64_t(3 * w + k) << 32 | uint64_t(tb + 9 * bb + k));
        }
      }
      std::sort(keys.begin(), keys.end());
      int32_t u = 0;
      uint64_t last = ~uint64_t(0);
      for (uint64_t key : keys)
        if ((key >> 32) != last) {
          last = key >> 32;
          ++u;
        }
      uniq[v] = u;
      for (int i = 0; i < 3; ++i) {  // row 3v + i: triplet ids shift by 3i
        const int64_t r = 3 * v + i;
        if (fx[r]) continue;
        int64_t q = rp[r];
        for (uint64_t key : keys) {
          x_col[q] = int32_t(key >> 32);
          ssrc[q] = int32_t(uint32_t(key) + 3u * uint32_t(i));
          ++q;
        }
      }
    }
  });
  // slots: a free row has its node's distinct columns, a fixed row one
  std::vector<int64_t> sp(n + 1, 0);
  for (int64_t r = 0; r < n; ++r) sp[r + 1] = sp[r] + (fx[r] ? 1 : uniq[r / 3]);
  const int64_t nnz = sp[n];
  if (nnz >= (int64_t(1) << 31)) return set_error(c, FE_ERR_ARG, "nnz exceeds int32");
  c->nnz = nnz;
  c->rowptr.resize(n + 1);
  for (int64_t r = 0; r <= n; ++r) c->rowptr[r] = int32_t(sp[r]);
  c->colind.assign(nnz, 0);
  c->slot_ptr.assign(nnz + 1, 0);
  c->C.assign(c->ntrip, -1);
  int32_t *colind = c->colind.data(), *Cm = c->C.data();
  int64_t *sptr = c->slot_ptr.data();
  parallel_chunks(n, 1536, [&](int64_t r0, int64_t r1) {
    for (int64_t r = r0; r < r1; ++r) {
      int64_t s = sp[r];
      if (fx[r]) {  // projected row: lone diagonal, no triplet maps to it
        colind[s] = int32_t(r);
        sptr[s] = rp[r];
        continue;
      }
      --s;
      int32_t last = -1;
      for (int64_t q = rp[r]; q < rp[r + 1]; ++q) {
        if (x_col[q] != last) {
          last = x_col[q];
          ++s;
          colind[s] = last;
          sptr[s] = q;
        }
        Cm[ssrc[q]] = int32_t(s);
      }
    }
  });
  sptr[nnz] = kept;
  return FE_OK;
}

// --------------------------------------------------------- mass, rest data
int build_mass_and_rest(fe_ctx *c) {
  const int npe = c->npe;
  const int64_t E = c->n_elems;
  const double *X = c->X.data();
  std::vector<double> me(size_t(E) * npe * npe);  // scalar consistent-mass blocks
  if (c->elem_type == FE_TET4) {
    c->rest_ncoef = 10;  // Dm^{-1} rows (grad N_1..3), volume
    c->rest.assign(size_t(10) * E, 0.0);
    for (int64_t e = 0; e < E; ++e) {
      const int32_t *cn = &c->conn[e * 4];
      double Dm[9];
      for (int i = 0; i < 3; ++i)
        for (int col = 0; col < 3; ++col) Dm[3 * i + col] = X[3 * cn[col + 1] + i] - X[3 * cn[0] + i];
      double V = det3(Dm) / 6.0;
      if (!(V > 0)) return set_error(c, FE_ERR_INVERTED, "tet " + std::to_string(e) + " has non-positive rest volume");
      double G[9];
      inv3(Dm, G);
      for (int k = 0; k < 9; ++k) c->rest[size_t(k) * E + e] = G[k];
      c->rest[size_t(9) * E + e] = V;
      for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) me[(e * 4 + a) * 4 + b] = c->rho * V / 20.0 * (a == b ? 2.0 : 1.0);
    }
  } else {
    c->rest_ncoef = 200;  // per Gauss point: grad N (8 x 3), w det J0
    c->rest.assign(size_t(200) * E, 0.0);
    for (int64_t e = 0; e < E; ++e) {
      const int32_t *cn = &c->conn[e * 8];
      for (int a = 0; a < 64; ++a) me[e * 64 + a] = 0.0;
      for (int q = 0; q < 8; ++q) {
        double xi[3], N[8], dN[8][3];
        hex_gauss(q, xi);
        hex_dshape(xi, N, dN);
        double J0[9] = {0};
        for (int a = 0; a < 8; ++a)
          for (int i = 0; i < 3; ++i)
            for (int r = 0; r < 3; ++r) J0[3 * i + r] += X[3 * cn[a] + i] * dN[a][r];
        double dj = det3(J0);
        if (!(dj > 0)) return set_error(c, FE_ERR_INVERTED, "hex " + std::to_string(e) + " has non-positive rest Jacobian");
        double Ji[9];
        inv3(J0, Ji);
        for (int a = 0; a < 8; ++a)
          for (int J = 0; J < 3; ++J) {
            double g = 0;
            for (int r = 0; r < 3; ++r) g += dN[a][r] * Ji[3 * r + J];
            c->rest[size_t(q * 25 + 3 * a + J) * E + e] = g;
          }
        c->rest[size_t(q * 25 + 24) * E + e] = dj;
        for (int a = 0; a < 8; ++a)
          for (int b = 0; b < 8; ++b) me[e * 64 + a * 8 + b] += c->rho * dj * N[a] * N[b];
      }
    }
  }
  // mass values on the pattern: gather through the inverse map (ascending t)
  c->mass.assign(c->nnz, 0.0);
  const int64_t bpe = int64_t(npe) * npe * 9;
  // slots in parallel; each slot sums its triplets in ascending order
  parallel_chunks(c->nnz, 4096, [&](int64_t s0, int64_t s1) {
    for (int64_t s = s0; s < s1; ++s) {
      double acc = 0.0;
      for (int64_t q = c->slot_ptr[s]; q < c->slot_ptr[s + 1]; ++q) {
        int64_t t = c->slot_src[q];
        int64_t e = t / bpe, r = t % bpe;
        int blk = int(r / 9), ik = int(r % 9);
        if (ik / 3 == ik % 3) acc += me[e * npe * npe + blk];
      }
      c->mass[s] = acc;
    }
  });
  // (the node incidence lists for the force gather come from build_csr)
  return FE_OK;
}

// ------------------------------------------------------ node-block view
// Every free node's three rows share one column structure (whole nodes are
// fixed), so the pattern is a set of 3x3 node blocks and the 9 slots of a
// block gather the same element blocks (e, a, b), whose 9 values are
// contiguous in K_e.  The block lists come from the (0, 0) slot of each block.
int build_blocks(fe_ctx *c) {
  const int64_t nn = c->n_nodes;
  c->bptr.assign(nn + 1, 0);
  c->bcol.clear();
  c->bsrc_ptr.clear();
  c->bsrc.clear();
  c->bmass.clear();
  for (int64_t v = 0; v < nn; ++v) {
    c->bptr[v] = int32_t(c->bcol.size());
    const int64_t r0 = 3 * v;
    if (c->fixed_dof[r0]) continue;
    const int32_t s0 = c->rowptr[r0], s1 = c->rowptr[r0 + 1];
    if ((s1 - s0) % 3 != 0) return set_error(c, FE_ERR_ARG, "row length not a multiple of 3");
    for (int32_t s = s0; s < s1; s += 3) {
      c->bcol.push_back(c->colind[s] / 3);
      c->bsrc_ptr.push_back(int32_t(c->bsrc.size()));
      for (int64_t q = c->slot_ptr[s]; q < c->slot_ptr[s + 1]; ++q) c->bsrc.push_back(c->slot_src[q] / 9);
      c->bmass.push_back(c->mass[s]);
    }
  }
  c->bptr[nn] = int32_t(c->bcol.size());
  c->bsrc_ptr.push_back(int32_t(c->bsrc.size()));
  return FE_OK;
}

// ------------------------------------------------------- nested dissection
struct ND {
  fe_ctx *c;
  std::vector<std::vector<int32_t>> adj;   // free-node graph
  std::vector<int32_t> order;              // new node position -> node
  std::vector<int32_t> tag;
  int32_t stamp = 0;
  int leaf = 64;
  struct F { int32_t first, count, parent = -1; std::vector<int32_t> kids; };
  std::vector<F> fr;

  int32_t make_front(std::vector<int32_t> &S) {
    std::sort(S.begin(), S.end());
    F f;
    f.first = int32_t(order.size());
    f.count = int32_t(S.size());
    order.insert(order.end(), S.begin(), S.end());
    fr.push_back(f);
    return int32_t(fr.size() - 1);
  }

  std::vector<int32_t> build(std::vector<int32_t> S) {
    if (S.empty()) return {};
    if (int(S.size()) <= leaf) return {make_front(S)};
    // longest axis of the rest bounding box
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int32_t v : S)
      for (int d = 0; d < 3; ++d) {
        lo[d] = std::min(lo[d], c->X[3 * v + d]);
        hi[d] = std::max(hi[d], c->X[3 * v + d]);
      }
    int ax = 0;
    for (int d = 1; d < 3; ++d)
      if (hi[d] - lo[d] > hi[ax] - lo[ax]) ax = d;
    std::vector<std::pair<double, int32_t>> key(S.size());
    for (size_t i = 0; i < S.size(); ++i) key[i] = {c->X[3 * S[i] + ax], S[i]};
    std::sort(key.begin(), key.end());
    // split at the widest coordinate gap near the median (a grid layer boundary)
    int64_t N = int64_t(S.size()), mid = N / 2, w = std::max<int64_t>(1, N / 8);
    int64_t best = mid;
    double bgap = -1.0;
    for (int64_t s = std::max<int64_t>(1, mid - w); s <= std::min<int64_t>(N - 1, mid + w); ++s) {
      double g = key[s].first - key[s - 1].first;
      if (g > bgap + 1e-15 * (std::fabs(key[s].first) + 1) ||
          (std::fabs(g - bgap) <= 1e-15 * (std::fabs(key[s].first) + 1) &&
           std::llabs(s - mid) < std::llabs(best - mid))) {
        bgap = g;
        best = s;
      }
    }
    // side tags: 1 = left, 2 = right
    int32_t sL = ++stamp, sR = ++stamp;
    for (int64_t i = 0; i < N; ++i) tag[key[i].second] = (i < best) ? sL : sR;
    std::vector<int32_t> bL, bR, L, R;
    for (int64_t i = 0; i < N; ++i) {
      int32_t v = key[i].second;
      int32_t other = (i < best) ? sR : sL;
      bool touch = false;
      for (int32_t u : adj[v])
        if (tag[u] == other) { touch = true; break; }
      if (i < best) { L.push_back(v); if (touch) bL.push_back(v); }
      else { R.push_back(v); if (touch) bR.push_back(v); }
    }
    std::vector<int32_t> sep, L2, R2;
    if (bR.size() <= bL.size()) {
      sep = bR;
      int32_t ss = ++stamp;
      for (int32_t v : sep) tag[v] = ss;
      L2 = L;
      for (int32_t v : R) if (tag[v] != ss) R2.push_back(v);
    } else {
      sep = bL;
      int32_t ss = ++stamp;
      for (int32_t v : sep) tag[v] = ss;
      R2 = R;
      for (int32_t v : L) if (tag[v] != ss) L2.push_back(v);
    }
    if (L2.empty() && R2.empty()) return {make_front(S)};
    std::vector<int32_t> kids = build(L2);
    std::vector<int32_t> kr = build(R2);
    kids.insert(kids.end(), kr.begin(), kr.end());
    if (sep.empty()) return kids;  // disconnected halves: independent subtrees
    int32_t f = make_front(sep);
    for (int32_t k : kids) { fr[k].parent = f; fr[f].kids.push_back(k); }
    return {f};
  }
};

int build_ordering(fe_ctx *c) {
  const int npe = c->npe;
  const int64_t nn = c->n_nodes;
  std::vector<int8_t> fixed_node(nn, 0);
  for (int32_t v : c->fixed_nodes) fixed_node[v] = 1;
  ND nd;
  nd.c = c;
  nd.leaf = c->opt.nd_leaf_nodes > 0 ? c->opt.nd_leaf_nodes : 64;
  nd.adj.assign(nn, {});
  for (int64_t e = 0; e < c->n_elems; ++e)
    for (int a = 0; a < npe; ++a) {
      int32_t va = c->conn[e * npe + a];
      if (fixed_node[va]) continue;
      for (int b = 0; b < npe; ++b) {
        int32_t vb = c->conn[e * npe + b];
        if (b != a && !fixed_node[vb]) nd.adj[va].push_back(vb);
      }
    }
  for (auto &l : nd.adj) {
    std::sort(l.begin(), l.end());
    l.erase(std::unique(l.begin(), l.end()), l.end());
  }
  nd.tag.assign(nn, 0);
  // one dissection per batch member: members share no edge, and their
  // coordinates overlap, so a joint geometric bisection would cut them all
  // with one shared separator; each member's tree is a root of the forest
  for (int32_t k = 0; k < c->nseg; ++k) {
    std::vector<int32_t> S;
    for (int64_t v = c->seg_node[k]; v < c->seg_node[k + 1]; ++v)
      if (!fixed_node[v]) S.push_back(int32_t(v));
    nd.build(S);
  }
  const int64_t nfree_nodes = int64_t(nd.order.size());
  std::vector<int32_t> pos(nn, -1);
  for (int64_t i = 0; i < nfree_nodes; ++i) pos[nd.order[i]] = int32_t(i);

  // DOF permutation: new DOF 3*pos + comp <-> original 3*node + comp
  c->n_free = 3 * nfree_nodes;
  c->perm.assign(c->n_free, 0);
  c->iperm.assign(c->n, -1);
  for (int64_t i = 0; i < nfree_nodes; ++i)
    for (int k = 0; k < 3; ++k) {
      c->perm[3 * i + k] = 3 * nd.order[i] + k;
      c->iperm[3 * nd.order[i] + k] = int32_t(3 * i + k);
    }

  // multifrontal symbolic analysis on nodes (fronts are in postorder)
  const int64_t nf = int64_t(nd.fr.size());
  std::vector<std::vector<int32_t>> upd(nf);  // update node positions, ascending
  std::vector<int32_t> mark(nfree_nodes, -1);
  for (int64_t f = 0; f < nf; ++f) {
    const auto &F = nd.fr[f];
    int32_t last = F.first + F.count - 1;
    std::vector<int32_t> &U = upd[f];
    for (int32_t i = F.first; i <= last; ++i)
      for (int32_t u : nd.adj[nd.order[i]]) {
        int32_t pu = pos[u];
        if (pu > last && mark[pu] != f) { mark[pu] = int32_t(f); U.push_back(pu); }
      }
    for (int32_t k : F.kids)
      for (int32_t pu : upd[k])
        if (pu > last && mark[pu] != f) { mark[pu] = int32_t(f); U.push_back(pu); }
    std::sort(U.begin(), U.end());
  }
  c->fronts.assign(nf, Front());
  c->y_nnz = 0;
  int64_t f_total = 0, y_total = 0, w_total = 0, u_total = 0, rows_total = 0;
  for (int64_t f = 0; f < nf; ++f) {
    Front &F = c->fronts[f];
    F.first = 3 * nd.fr[f].first;
    F.npiv = 3 * nd.fr[f].count;
    F.nupd = 3 * int32_t(upd[f].size());
    F.parent = nd.fr[f].parent;
    int lv = 0;
    for (int32_t k : nd.fr[f].kids) lv = std::max(lv, c->fronts[k].level + 1);
    F.level = lv;
    int64_t m = F.m();
    F.ldy = int32_t((m + 7) / 8 * 8);  // 16-byte vectors of binary16 entries stay aligned
    F.ldf = int32_t((m + 3) / 4 * 4);
    F.f_off = f_total; f_total += int64_t(F.ldf) * m;
    F.y_off = y_total; y_total += int64_t(F.ldy) * F.npiv;
    F.w_off = w_total; w_total += m;
    F.u_off = u_total; u_total += F.nupd;
    F.rows_off = rows_total; rows_total += F.nupd;
    c->y_nnz += m * F.npiv - int64_t(F.npiv) * (F.npiv - 1) / 2;
  }
  c->f_total = f_total; c->y_total = y_total; c->w_total = w_total; c->u_total = u_total;
  c->upd_rows_new.assign(rows_total, 0);
  c->upd_rows_old.assign(rows_total, 0);
  for (int64_t f = 0; f < nf; ++f) {
    const Front &F = c->fronts[f];
    for (size_t j = 0; j < upd[f].size(); ++j)
      for (int k = 0; k < 3; ++k) {
        int32_t nw = 3 * upd[f][j] + k;
        c->upd_rows_new[F.rows_off + 3 * j + k] = nw;
        c->upd_rows_old[F.rows_off + 3 * j + k] = c->perm[nw];
      }
  }
  // children lists and child -> parent relative maps
  c->child_ptr.assign(nf + 1, 0);
  for (int64_t f = 0; f < nf; ++f) c->child_ptr[f + 1] = int32_t(nd.fr[f].kids.size());
  for (int64_t f = 0; f < nf; ++f) c->child_ptr[f + 1] += c->child_ptr[f];
  c->child_list.assign(c->child_ptr[nf], 0);
  for (int64_t f = 0; f < nf; ++f)
    for (size_t k = 0; k < nd.fr[f].kids.size(); ++k) c->child_list[c->child_ptr[f] + k] = nd.fr[f].kids[k];
  c->rmap.assign(rows_total, 0);
  for (int64_t f = 0; f < nf; ++f) {
    Front &F = c->fronts[f];
    F.rmap_off = F.rows_off;
    if (F.parent < 0) continue;
    const Front &P = c->fronts[F.parent];
    const int32_t *prow = &c->upd_rows_new[P.rows_off];
    for (int32_t j = 0; j < F.nupd; ++j) {
      int32_t nw = c->upd_rows_new[F.rows_off + j];
      int32_t loc;
      if (nw >= P.first && nw < P.first + P.npiv) {
        loc = nw - P.first;
      } else {
        const int32_t *it = std::lower_bound(prow, prow + P.nupd, nw);
        if (it == prow + P.nupd || *it != nw)
          return set_error(c, FE_ERR_ARG, "symbolic analysis: update row missing in parent");
        loc = P.npiv + int32_t(it - prow);
      }
      c->rmap[F.rows_off + j] = loc;
    }
  }
  // gather lists of the forward apply: front position -> children's update entries
  {
    std::vector<std::vector<int32_t>> lists(w_total);
    for (int64_t f = 0; f < nf; ++f)
      for (int32_t k : nd.fr[f].kids) {
        const Front &Ch = c->fronts[k];
        for (int32_t j = 0; j < Ch.nupd; ++j)
          lists[c->fronts[f].w_off + c->rmap[Ch.rows_off + j]].push_back(int32_t(Ch.u_off + j));
      }
    c->wsrc_ptr.assign(w_total + 1, 0);
    c->wsrc.clear();
    for (int64_t q = 0; q < w_total; ++q) {
      c->wsrc_ptr[q] = int32_t(c->wsrc.size());
      c->wsrc.insert(c->wsrc.end(), lists[q].begin(), lists[q].end());
    }
    c->wsrc_ptr[w_total] = int32_t(c->wsrc.size());
  }
  // A entries of every front (lower triangle in the new order), by column
  c->fa_ptr.assign(nf + 1, 0);
  c->fa_slot.clear();
  c->fa_off.clear();
  c->fa_colptr.clear();
  for (int64_t f = 0; f < nf; ++f) {
    const Front &F = c->fronts[f];
    const int32_t *prow = &c->upd_rows_new[F.rows_off];
    c->fa_ptr[f] = int64_t(c->fa_slot.size());
    for (int32_t jl = 0; jl < F.npiv; ++jl) {
      c->fa_colptr.push_back(int64_t(c->fa_slot.size()));
      int32_t jn = F.first + jl, jo = c->perm[jn];
      for (int32_t k = c->rowptr[jo]; k < c->rowptr[jo + 1]; ++k) {
        int32_t in = c->iperm[c->colind[k]];
        if (in < jn) continue;
        int32_t lr;
        if (in < F.first + F.npiv) {
          lr = in - F.first;
        } else {
          const int32_t *it = std::lower_bound(prow, prow + F.nupd, in);
          if (it == prow + F.nupd || *it != in)
            return set_error(c, FE_ERR_ARG, "symbolic analysis: A entry outside its front");
          lr = F.npiv + int32_t(it - prow);
        }
        c->fa_slot.push_back(k);
        c->fa_off.push_back(lr + jl * F.ldf);
      }
    }
    c->fa_colptr.push_back(int64_t(c->fa_slot.size()));
  }
  c->fa_ptr[nf] = int64_t(c->fa_slot.size());
  if (c->f_total >= (int64_t(1) << 40)) return set_error(c, FE_ERR_OOM, "front storage too large");

  // public views
  c->front_first.resize(nf); c->front_npiv.resize(nf); c->front_nupd.resize(nf);
  c->front_parent.resize(nf); c->front_level.resize(nf);
  int maxlv = 0;
  for (int64_t f = 0; f < nf; ++f) {
    c->front_first[f] = c->fronts[f].first;
    c->front_npiv[f] = c->fronts[f].npiv;
    c->front_nupd[f] = c->fronts[f].nupd;
    c->front_parent[f] = c->fronts[f].parent;
    c->front_level[f] = c->fronts[f].level;
    maxlv = std::max(maxlv, c->fronts[f].level);
  }

  // level schedule and static task lists
  c->levels.assign(nf ? maxlv + 1 : 0, Level());
  for (int64_t f = 0; f < nf; ++f) c->levels[c->fronts[f].level].fronts.push_back(int32_t(f));
  double flops = 0;
  // trailing-update tile: 128 x 128 for the FP32 factor, 64 x 64 for FP64
  const int32_t ut = c->opt.precision == FE_MIXED ? 128 : kTile;
  const int32_t sp = c->opt.precision == FE_MIXED ? kSuper : kNB;
  // the superpanels' deferred updates go to the BF16 kernel's lists
  const bool bf16_end = c->opt.precision == FE_MIXED && c->opt.update_bf16;
  const int32_t fr_rows = fwd_rows(c->opt);
  const int32_t vw = y_vec(c->opt);  // rows per 16-byte vector of Y
  const int32_t br = bwd_rows(c->opt);
  c->fwd_slots = c->bwd_slots = 0;
  for (auto &L : c->levels) {
    int steps = 0;
    for (int32_t f : L.fronts) steps = std::max(steps, (c->fronts[f].npiv + kNB - 1) / kNB);
    L.steps = steps;
    L.diag.assign(steps, {});
    L.panel.assign(steps, {});
    L.trail.assign(steps, {});
    L.trail_flops.assign(steps, 0.0);
    L.tend.assign(steps, {});
    L.tend_flops.assign(steps, 0.0);
    // assembly tasks: narrower column ranges for larger fronts (a task's
    // work grows with the front's rows; the top levels hold few fronts), the
    // largest fronts first so that the level's last wave is short
    {
      std::vector<int32_t> order(L.fronts);
      std::stable_sort(order.begin(), order.end(),
                       [&](int32_t a, int32_t b) { return c->fronts[a].m() > c->fronts[b].m(); });
      for (int32_t f : order) {
        const int32_t m = c->fronts[f].m();
        const int32_t w = m > 2048 ? 8 : m > 1024 ? 16 : 32;
        for (int32_t c0 = 0; c0 < m; c0 += w) {
          L.asm_tasks.push_back(f);
          L.asm_tasks.push_back(c0);
          L.asm_tasks.push_back(std::min(m, c0 + w));
        }
      }
    }
    // task sizes of the application sweeps on this level: a level with
    // fewer than kApplyTasksPerLevel tasks at the full sizes (the few large
    // fronts near the root) takes narrower ones, down to a quarter, so its
    // dependency chain spreads over more CTAs
    auto fwd_count = [&](int32_t fc) {
      int64_t n = 0;
      for (int32_t f : L.fronts) {
        const Front &F = c->fronts[f];
        for (int32_t r0 = 0; r0 < F.m(); r0 += fr_rows) n += std::max(1, (std::min(r0 + fr_rows, F.npiv) + fc - 1) / fc);
      }
      return n;
    };
    auto bwd_count = [&](int32_t b) {
      int64_t n = 0;
      for (int32_t f : L.fronts) {
        const Front &F = c->fronts[f];
        for (int32_t c0 = 0; c0 < F.npiv; c0 += kBwdCols) n += (F.ldy - 1) / b - (c0 & ~(vw - 1)) / b + 1;
      }
      return n;
    };
    int32_t lfc = kFwdCols, lbr = br;
    while (lfc > kFwdCols / 4 && fwd_count(lfc) < kApplyTasksPerLevel) lfc /= 2;
    while (lbr > br / 4 && lbr / 2 >= vw && bwd_count(lbr) < kApplyTasksPerLevel) lbr /= 2;
    for (int32_t f : L.fronts) {
      c->fronts[f].fcols = lfc;
      c->fronts[f].brows = lbr;
      const Front &F = c->fronts[f];
      const int32_t m = F.m(), p = F.npiv;
      // apply tasks; a block split over several tasks owns consecutive
      // partial-sum slots, reduced in order by the last task to finish
      for (int32_t r0 = 0; r0 < m; r0 += fr_rows) {
        const int32_t jmax = std::min(r0 + fr_rows, p);
        const int32_t nch = std::max(1, (jmax + lfc - 1) / lfc);
        const int32_t slot = nch > 1 ? int32_t(c->fwd_slots) : -1;
        if (nch > 1) c->fwd_slots += nch;
        for (int32_t k = 0; k < nch; ++k) {
          L.fwd_tasks.push_back(f); L.fwd_tasks.push_back(r0);
          L.fwd_tasks.push_back(k * lfc); L.fwd_tasks.push_back(slot);
        }
      }
      for (int32_t c0 = 0; c0 < p; c0 += kBwdCols) {
        const int32_t a0 = c0 & ~(vw - 1);
        const int32_t k0 = a0 / lbr, k1 = (F.ldy - 1) / lbr;
        const int32_t slot = k1 > k0 ? int32_t(c->bwd_slots) : -1;
        if (k1 > k0) c->bwd_slots += k1 - k0 + 1;
        for (int32_t k = k0; k <= k1; ++k) {
          L.bwd_tasks.push_back(f); L.bwd_tasks.push_back(c0);
          L.bwd_tasks.push_back(k * lbr); L.bwd_tasks.push_back(slot);
        }
      }
      for (int s = 0; s * kNB < p; ++s) {
        const int32_t k0 = s * kNB, kb = std::min(kNB, p - k0), k1 = k0 + kb;
        auto push = [](std::vector<int32_t> &v, int32_t a, int32_t b, int32_t cc, int32_t d) {
          v.push_back(a); v.push_back(b); v.push_back(cc); v.push_back(d);
        };
        push(L.diag[s], f, (T_DIAG << 24) | k0, kb, 0);
        for (int32_t r0 = k1; r0 < m; r0 += kTile) push(L.panel[s], f, (T_PANEL << 24) | k0, r0, 0);
        for (int32_t c0 = 0; c0 < k0; c0 += kTile) push(L.panel[s], f, (T_XK << 24) | k0, c0, 0);
        // trailing and Y updates (FP32 path): eager inside the sub-block
        // [b0, b1) of the superpanel [s0, s1), the rest of the superpanel's
        // columns (rows of Y) once per sub-block with K = b1 - b0, the rest
        // of the front once per superpanel with K = s1 - s0
        const int32_t s0 = k0 / sp * sp, s1 = std::min(s0 + sp, p);
        const int32_t sb = std::min(kSub, sp);
        const int32_t b0 = k0 / sb * sb, b1 = std::min(b0 + sb, s1);
        for (int32_t j0 = k1; j0 < b1; j0 += ut)
          for (int32_t i0 = j0; i0 < m; i0 += ut) push(L.trail[s], f, (T_TRAIL << 24) | k0, i0, j0);
        for (int32_t i0 = k1; i0 < b1; i0 += ut)
          for (int32_t c0 = 0; c0 < k1; c0 += ut) push(L.trail[s], f, (T_RUPD << 24) | k0, i0, c0);
        if (k1 == b1 && b1 < s1) {
          // b1 is a multiple of kSub here, so the tiles start aligned
          const int32_t chunks = (b1 - b0 + kNB - 1) / kNB;
          const int32_t code = ((T_TRAIL | ((chunks - 1) << 3)) << 24) | b0;
          const int32_t codeu = ((T_RUPD | ((chunks - 1) << 3)) << 24) | b0;
          for (int32_t j0 = b1; j0 < s1; j0 += ut)
            for (int32_t i0 = j0; i0 < m; i0 += ut) push(L.trail[s], f, code, i0, j0);
          for (int32_t i0 = b1; i0 < s1; i0 += ut)
            for (int32_t c0 = 0; c0 < b1; c0 += ut) push(L.trail[s], f, codeu, i0, c0);
        }
        if (k1 == s1) {
          const int32_t chunks = (s1 - s0 + kNB - 1) / kNB;
          const int32_t code = ((T_TRAIL | ((chunks - 1) << 3)) << 24) | s0;
          const int32_t codeu = ((T_RUPD | ((chunks - 1) << 3)) << 24) | s0;
          // FP32 path: tiles start at a multiple of 4 rows (a TMA box must
          // start 16-byte aligned); the rows and columns of the tile below
          // s1 belong to the superpanel and are left alone by the kernel
          const int32_t t1 = c->opt.precision == FE_MIXED ? (s1 & ~3) : s1;
          auto &dst = bf16_end ? L.tend[s] : L.trail[s];
          for (int32_t j0 = t1; j0 < m; j0 += ut)
            for (int32_t i0 = j0; i0 < m; i0 += ut) push(dst, f, code, i0, j0);
          for (int32_t i0 = t1; i0 < m; i0 += ut)
            for (int32_t c0 = 0; c0 < s1; c0 += ut) push(dst, f, codeu, i0, c0);
        }
        // algorithmic flops of this panel's updates (the zero products of the
        // superpanel's upper triangle in Y are not counted); with the BF16
        // superpanel ends, the part applied there (rows and columns from the
        // superpanel's end s1 on) is booked to the end step
        const double rem = double(m - k1);
        const double all_flops = rem * (rem + 1.0) * kb + 2.0 * rem * double(k1) * kb;
        if (bf16_end) {
          const double re = double(m - s1);
          const double end_flops = re * (re + 1.0) * kb + 2.0 * re * double(k1) * kb;
          const int s_end_step = (s1 - 1) / kNB;
          L.trail_flops[s] += all_flops - end_flops;
          L.tend_flops[s_end_step] += end_flops;
        } else {
          L.trail_flops[s] += all_flops;
        }
        flops += double(kb) * kb * kb / 3.0 * 2.0            // diag LDL^T + inverse
                 + 2.0 * rem * kb * kb                        // panel
                 + 2.0 * double(kb) * kb * k0                 // X_K
                 + rem * (rem + 1.0) * kb                     // trailing (lower)
                 + 2.0 * rem * double(k1) * kb;               // Y update
      }
    }
  }
  c->factor_flops = flops;
  c->apply_fwd.clear();
  c->apply_bwd.clear();
  c->front_nfwd.assign(nf, 0);
  c->front_nbwd.assign(nf, 0);
  for (const auto &L : c->levels) {
    c->apply_fwd.insert(c->apply_fwd.end(), L.fwd_tasks.begin(), L.fwd_tasks.end());
    for (size_t k = 0; k < L.fwd_tasks.size(); k += 4) c->front_nfwd[L.fwd_tasks[k]]++;
  }
  for (size_t lv = c->levels.size(); lv-- > 0;) {
    const auto &L = c->levels[lv];
    c->apply_bwd.insert(c->apply_bwd.end(), L.bwd_tasks.begin(), L.bwd_tasks.end());
    for (size_t k = 0; k < L.bwd_tasks.size(); k += 4) c->front_nbwd[L.bwd_tasks[k]]++;
  }
  return FE_OK;
}

}  // namespace

int build_pattern_host(fe_ctx *c) {
  c->n = 3 * c->n_nodes;
  c->fixed_dof.assign(c->n, 0);
  for (int32_t v : c->fixed_nodes)
    for (int k = 0; k < 3; ++k) c->fixed_dof[3 * int64_t(v) + k] = 1;
  int st = build_csr(c);
  if (st) return st;
  st = build_mass_and_rest(c);
  if (st) return st;
  st = build_blocks(c);
  if (st) return st;
  st = build_ordering(c);
  if (st) return st;
  c->built = true;
  return FE_OK;
}

}  // namespace fe
