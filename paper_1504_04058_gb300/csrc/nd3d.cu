// nd3d.cu -- the 3D slab subproblems H_q^M, H_p^R, H_p^L by nested dissection
// (Section 4: the unknowns of a quasi-2D slab are grouped along dimension 3 and
// the grouped problem is ordered by nested dissection; Algorithm 3 builds the
// factorizations, Algorithm 4 applies them).
//
// Ordering.  A slab of width w has n x n columns (i1, i2) of w unknowns each.
// The column grid is cut recursively: a region of more than kNdLeafCols columns
// is split by the middle line across its longer side (the separator: the line's
// columns, all w planes), and each half is cut again; a region of at most
// kNdLeafCols columns is a leaf whose unknowns are all its columns.  Node t
// owns the unknowns I(t) (its separator, or a leaf's region); its boundary B(t)
// is the columns just outside its region (4-neighbours across its sides), which
// lie on separators of its ancestors.  The tree depends on n only.
//
// Factorization (multifrontal, explicit inverses).  Bottom-up, level by level,
// every node's front F = [F_II F_IB; F_BI F_BB] (rows and columns I(t) then
// B(t), w planes per column, planes fastest) is assembled from the stencil
// entries coupling I(t) to I(t) u B(t) plus the update matrices of its children
// (extend-add).  Gauss-Jordan steps on the I columns, with pivots searched in the
// I rows only, leave X = F_II^-1, X F_IB, -F_BI X and the Schur complement
// U = F_BB - F_BI X F_IB in the front (factor3d.cu's blocked engine with
// np = |I|; at complex64 the levels whose fronts reach kNdTcMinFront unknowns
// run its rank-256 updates on the tensor cores, tcupdate.cu).  Stored: [X; L] with L = F_BI X, and P = X F_IB; U passes to the
// parent.
//
// Solve.  Forward (leaves to root): f_I = g restricted to I(t) plus the
// children's update vectors on I(t), f_B = the children's update vectors on
// B(t); z = X f_I; u = f_B - L f_I goes to the parent.  Backward (root to
// leaves): x_I = z - P x_B, with x_B the ancestors' values already solved.
// Every launch covers one tree depth for a batch of slab solves; the update
// vectors move through per-front scratch, so no two CTAs write one address.
#include <algorithm>
#include <functional>
#include <string>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace asp {

// ------------------------------------------------------------------ plan
bool nd_build_tree(int n, NdTree& T, std::string* why) {
  T = NdTree();
  T.n = n;
  struct Tmp {
    int depth, parent, c0 = -1, c1 = -1;
    std::vector<int> icol, bcol;
  };
  std::vector<Tmp> v;
  std::function<int(int, int, int, int, int, int)> rec = [&](int x0, int x1, int y0, int y1, int depth,
                                                            int parent) -> int {
    const int id = (int)v.size();
    v.push_back(Tmp());
    v[id].depth = depth;
    v[id].parent = parent;
    std::vector<int> B, I;
    if (y0 > 0)
      for (int x = x0; x < x1; ++x) B.push_back((y0 - 1) * n + x);
    if (x0 > 0)
      for (int y = y0; y < y1; ++y) B.push_back(y * n + x0 - 1);
    if (x1 < n)
      for (int y = y0; y < y1; ++y) B.push_back(y * n + x1);
    if (y1 < n)
      for (int x = x0; x < x1; ++x) B.push_back(y1 * n + x);
    std::sort(B.begin(), B.end());
    const int W = x1 - x0, Hh = y1 - y0;
    int c0 = -1, c1 = -1;
    if (W * Hh <= kNdLeafCols) {
      for (int y = y0; y < y1; ++y)
        for (int x = x0; x < x1; ++x) I.push_back(y * n + x);
    } else if (W >= Hh) {  // W >= 5 here, so both halves are non-empty
      const int xs = (x0 + x1) / 2;
      for (int y = y0; y < y1; ++y) I.push_back(y * n + xs);
      c0 = rec(x0, xs, y0, y1, depth + 1, id);
      c1 = rec(xs + 1, x1, y0, y1, depth + 1, id);
    } else {
      const int ys = (y0 + y1) / 2;
      for (int x = x0; x < x1; ++x) I.push_back(ys * n + x);
      c0 = rec(x0, x1, y0, ys, depth + 1, id);
      c1 = rec(x0, x1, ys + 1, y1, depth + 1, id);
    }
    std::sort(I.begin(), I.end());
    v[id].icol = I;
    v[id].bcol = B;
    v[id].c0 = c0;
    v[id].c1 = c1;
    return id;
  };
  rec(0, n, 0, n, 0, -1);
  T.nn = (int)v.size();
  T.node.assign((size_t)T.nn * kNdNodeInts, 0);
  for (int t = 0; t < T.nn; ++t) {
    int* nd = &T.node[(size_t)t * kNdNodeInts];
    nd[ND_NCI] = (int)v[t].icol.size();
    nd[ND_NCB] = (int)v[t].bcol.size();
    nd[ND_OFFC] = (int)T.cols.size();
    T.cols.insert(T.cols.end(), v[t].icol.begin(), v[t].icol.end());
    T.cols.insert(T.cols.end(), v[t].bcol.begin(), v[t].bcol.end());
    nd[ND_C0] = v[t].c0;
    nd[ND_C1] = v[t].c1;
    nd[ND_DEPTH] = v[t].depth;
    T.maxdepth = std::max(T.maxdepth, v[t].depth);
    nd[ND_OFFM] = -1;
    if (v[t].parent >= 0) {
      const Tmp& P = v[v[t].parent];
      nd[ND_OFFM] = (int)T.cmap.size();
      for (int c : v[t].bcol) {
        auto it = std::lower_bound(P.icol.begin(), P.icol.end(), c);
        int pos = -1;
        if (it != P.icol.end() && *it == c) {
          pos = (int)(it - P.icol.begin());
        } else {
          auto jt = std::lower_bound(P.bcol.begin(), P.bcol.end(), c);
          if (jt != P.bcol.end() && *jt == c) pos = (int)P.icol.size() + (int)(jt - P.bcol.begin());
        }
        if (pos < 0) {
          if (why) *why = "nested dissection: a boundary column of a node is not in its parent's front";
          return false;
        }
        T.cmap.push_back(pos);
      }
    }
  }
  T.at_depth.assign(T.maxdepth + 1, std::vector<int>());
  for (int t = 0; t < T.nn; ++t) T.at_depth[v[t].depth].push_back(t);
  return true;
}

namespace {

inline int r4(int x) { return (x + 3) & ~3; }
// work elements of one front in the Gauss-Jordan engine's layout: the front,
// the outer block's pivot rows and the inner panel's pivot rows
inline long long front_work(int ns) {
  const int ld = r4(ns);
  return (long long)ns * ld + (long long)kSlabOuter * ld + (long long)kSlabPanel * kSlabOuter;
}
// work budget of one factor group (bytes; the two groups run concurrently)
constexpr long long kNdGroupWorkBytes = 8LL << 30;

}  // namespace

NdSizes nd_sizes(const NdTree& T, const std::vector<int>& widths, const std::vector<int>& kinds, int max_rhs,
                 int esz, std::vector<int>* chunk) {
  NdSizes Z;
  const int D = T.maxdepth + 1;
  // per width: each depth's work elements
  auto level_work = [&](int w) {
    std::vector<long long> lw(D, 0);
    for (int t = 0; t < T.nn; ++t) lw[T.node[t * kNdNodeInts + ND_DEPTH]] += front_work(T.nc(t) * w);
    return lw;
  };
  for (size_t i = 0; i < widths.size(); ++i) {
    const int w = widths[i];
    for (int t = 0; t < T.nn; ++t) {
      const int s = T.node[t * kNdNodeInts + ND_NCI] * w, B = T.node[t * kNdNodeInts + ND_NCB] * w;
      const int ns = s + B;
      Z.factor_elems += (long long)ns * r4(s) + (long long)s * r4(B);
      Z.piv_ints += 3LL * ns;
      Z.zu_elems += (long long)ns * max_rhs;
      Z.max_front = std::max(Z.max_front, ns);
      Z.nfronts++;
    }
  }
  if (chunk) chunk->assign(widths.size(), 0);
  std::vector<int> ckof(widths.size(), 0);
  // chunks per group (group 0: the M slabs; group 1: the R and L slabs),
  // greedily while both parity buffers stay inside the budget
  const long long budget = kNdGroupWorkBytes / esz;
  for (int g = 0; g < 2; ++g) {
    std::vector<long long> cur(D, 0);
    long long best0 = 0, best1 = 0;  // the group's largest even / odd depth buffer over its chunks
    int ck = 0;
    bool any = false;
    for (size_t i = 0; i < widths.size(); ++i) {
      if ((kinds[i] == KIND_M) != (g == 0)) continue;
      const std::vector<long long> lw = level_work(widths[i]);
      std::vector<long long> nxt(D);
      long long e0 = 0, e1 = 0;
      for (int d = 0; d < D; ++d) {
        nxt[d] = cur[d] + lw[d];
        if (d % 2) e1 = std::max(e1, nxt[d]);
        else e0 = std::max(e0, nxt[d]);
      }
      if (any && e0 + e1 > budget) {  // start a new chunk
        ++ck;
        std::fill(cur.begin(), cur.end(), 0);
        for (int d = 0; d < D; ++d) nxt[d] = lw[d];
        e0 = e1 = 0;
        for (int d = 0; d < D; ++d) {
          if (d % 2) e1 = std::max(e1, nxt[d]);
          else e0 = std::max(e0, nxt[d]);
        }
      }
      cur = nxt;
      any = true;
      best0 = std::max(best0, e0);
      best1 = std::max(best1, e1);
      if (chunk) (*chunk)[i] = ck;
      ckof[i] = ck;
    }
    Z.work_elems += best0 + best1;
    if (esz == 8) {  // complex64: operand rows (fronts padded to 128) of each large-front level
      long long best = 0;
      for (int c = 0; c <= ck; ++c)
        for (int d = 0; d < D; ++d) {
          long long rows = 0;
          int nbmax = 0;
          for (size_t i = 0; i < widths.size(); ++i) {
            if ((kinds[i] == KIND_M) != (g == 0) || ckof[i] != c) continue;
            for (int t : T.at_depth[d]) {
              const int ns = T.nc(t) * widths[i];
              nbmax = std::max(nbmax, ns);
              rows += (ns + 127) / 128 * 128;
            }
          }
          if (nbmax >= kNdTcMinFront) best = std::max(best, rows);
        }
      Z.tc_floats += tc_group_floats(best);
    }
  }
  return Z;
}

}  // namespace asp

// Host-only check of the nested-dissection plan of an n x n column grid with w
// planes (no device call).  stats (up to 9 entries): nodes, largest depth,
// largest front, factor entries, assembled stencil entries, the slab operator's
// number of nonzeros, stencil couplings assembled more than once, couplings
// never assembled, complex multiply-adds of the fronts' Gauss-Jordan steps.
extern "C" int asp_nd_plan_check(int n, int w, long long* stats, int nstats) {
  using namespace asp;
  if (n < 1 || w < 1 || (long long)n * n > (1LL << 26)) return fail(ASP_ERR_INVALID, "nd plan: bad n or w");
  NdTree T;
  std::string why;
  if (!nd_build_tree(n, T, &why)) return fail(ASP_ERR_INVALID, why);
  std::vector<int> widths(1, w), kinds(1, KIND_M);
  const NdSizes Z = nd_sizes(T, widths, kinds, 1, 8, nullptr);
  // every stencil coupling (u, v) of the slab is assembled at exactly one front:
  // rows of I(t) take their couplings into I(t) u B(t); rows of B(t) their
  // couplings into I(t).  Count each pair.
  const long long N = (long long)n * n * w;
  auto uid = [&](int col, int pl) { return (long long)col * w + pl; };
  std::vector<unsigned char> seen;  // per (unknown, direction 0..6)
  seen.assign((size_t)N * 7, 0);
  long long assembled = 0, dup = 0;
  auto mark = [&](long long u, int dir) {
    ++assembled;
    unsigned char& s = seen[(size_t)u * 7 + dir];
    if (s) ++dup;
    s = 1;
  };
  for (int t = 0; t < T.nn; ++t) {
    const int* nd = &T.node[(size_t)t * kNdNodeInts];
    const int ncI = nd[ND_NCI], ncB = nd[ND_NCB];
    const int* cI = &T.cols[nd[ND_OFFC]];
    const int* cB = cI + ncI;
    auto inI = [&](int c) { return std::binary_search(cI, cI + ncI, c); };
    auto inB = [&](int c) { return std::binary_search(cB, cB + ncB, c); };
    for (int a = 0; a < ncI + ncB; ++a) {
      const int col = a < ncI ? cI[a] : cB[a - ncI];
      const int i1 = col % n, i2 = col / n;
      const int nb[4] = {i1 > 0 ? col - 1 : -1, i1 < n - 1 ? col + 1 : -1, i2 > 0 ? col - n : -1,
                         i2 < n - 1 ? col + n : -1};
      for (int pl = 0; pl < w; ++pl) {
        const long long u = uid(col, pl);
        if (a < ncI) {
          mark(u, 0);
          if (pl > 0) mark(u, 5);
          if (pl < w - 1) mark(u, 6);
          for (int d = 0; d < 4; ++d)
            if (nb[d] >= 0 && (inI(nb[d]) || inB(nb[d]))) mark(u, 1 + d);
        } else {
          for (int d = 0; d < 4; ++d)
            if (nb[d] >= 0 && inI(nb[d])) mark(u, 1 + d);
        }
      }
    }
  }
  long long miss = 0;
  for (int col = 0; col < n * n; ++col) {
    const int i1 = col % n, i2 = col / n;
    const bool has[4] = {i1 > 0, i1 < n - 1, i2 > 0, i2 < n - 1};
    for (int pl = 0; pl < w; ++pl) {
      const long long u = uid(col, pl);
      if (!seen[(size_t)u * 7 + 0]) ++miss;
      if (pl > 0 && !seen[(size_t)u * 7 + 5]) ++miss;
      if (pl < w - 1 && !seen[(size_t)u * 7 + 6]) ++miss;
      for (int d = 0; d < 4; ++d)
        if (has[d] && !seen[(size_t)u * 7 + 1 + d]) ++miss;
    }
  }
  const long long nnz = N + 2LL * ((long long)(n - 1) * n * w + (long long)n * (n - 1) * w + (long long)n * n * (w - 1));
  long long gj = 0;  // s steps, each updating the ns x ns front
  for (int t = 0; t < T.nn; ++t) {
    const long long sI = (long long)T.node[(size_t)t * kNdNodeInts + ND_NCI] * w, ns = (long long)T.nc(t) * w;
    gj += sI * ns * ns;
  }
  const long long out[9] = {T.nn, T.maxdepth, Z.max_front, Z.factor_elems, assembled, nnz, dup, miss, gj};
  for (int i = 0; i < nstats && i < 9; ++i) stats[i] = out[i];
  return ASP_OK;
}

namespace asp {

namespace {

// The int table on the device: node table, then the columns, the child maps and
// the node lists per depth.
struct NdTab {
  const int* node;
  const int* cols;
  const int* cmap;
  int nn, n;
};

struct NdKParams {
  NdTab T;
  const NdFront* fr;
  const Slab* eslab;  // engine view of every front
  const Slab* slabs;  // the handle's slabs
  const int* list;    // fronts of this launch
  void* A;            // work area
  int* piv;
  void* W;            // factors
};

__device__ __forceinline__ int nd_find(const int* a, int len, int key) {
  int lo = 0, hi = len - 1;
  while (lo <= hi) {
    const int mid = (lo + hi) >> 1;
    const int v = a[mid];
    if (v == key) return mid;
    if (v < key) lo = mid + 1;
    else hi = mid - 1;
  }
  return -1;
}

// ------------------------------------------------------------ assembly
// Row r = blockIdx.x of front list[blockIdx.y]: zero it, then the stencil
// entries of A that are assembled at this front (rows of I(t): couplings into
// I(t) u B(t); rows of B(t): couplings into I(t)); row_step[r] = -1.
template <typename R>
__global__ void __launch_bounds__(256) nd_assemble_kernel(NdKParams K, FactorCoefs<R> F) {
  using C = Cx<R>;
  const int f = K.list[blockIdx.y];
  const Slab E = K.eslab[f];
  const int r = blockIdx.x;
  if (r >= E.nb) return;
  const NdFront fr = K.fr[f];
  const Slab S = K.slabs[fr.slab];
  const int* nd = K.T.node + fr.node * kNdNodeInts;
  const int ncI = nd[ND_NCI], ncB = nd[ND_NCB];
  const int* cI = K.T.cols + nd[ND_OFFC];
  const int* cB = cI + ncI;
  const int w = fr.w, n = K.T.n, ld = E.ld, s = E.np;
  C* row = reinterpret_cast<C*>(K.A) + E.aoff + (long long)r * ld;
  for (int j = threadIdx.x; j < ld; j += blockDim.x) row[j] = czero<R>();
  __syncthreads();
  if (threadIdx.x != 0) return;
  K.piv[E.poff + 2LL * E.nb + r] = -1;
  const int ci = r / w, i3l = r - ci * w;
  const int col = ci < ncI ? cI[ci] : cB[ci - ncI];
  const int i1 = col % n, i2 = col / n;
  const int nbc[4] = {i1 > 0 ? col - 1 : -1, i1 < n - 1 ? col + 1 : -1, i2 > 0 ? col - n : -1,
                      i2 < n - 1 ? col + n : -1};
  const C cf[4] = {F.ca[i1], F.cc[i1], F.ca[i2], F.cc[i2]};
  if (r < s) {
    C diag = cadd(cadd(F.dg[S.prof + i3l], F.cd[i1]), F.cd[i2]);
    diag.x += F.k2[((long long)(S.lo - 1 + i3l) * n + i2) * n + i1];
    row[r] = diag;
    if (i3l > 0) row[r - 1] = F.dn[S.prof + i3l];
    if (i3l < w - 1) row[r + 1] = F.up[S.prof + i3l];
    for (int d = 0; d < 4; ++d) {
      if (nbc[d] < 0) continue;
      int p = nd_find(cI, ncI, nbc[d]);
      if (p < 0) {
        p = nd_find(cB, ncB, nbc[d]);
        if (p >= 0) p += ncI;
      }
      if (p >= 0) row[p * w + i3l] = cf[d];
    }
  } else {
    for (int d = 0; d < 4; ++d) {
      if (nbc[d] < 0) continue;
      const int p = nd_find(cI, ncI, nbc[d]);
      if (p >= 0) row[p * w + i3l] = cf[d];
    }
  }
}

// Extend-add of child `slot` of every front of the list: row b = blockIdx.x of
// the child's update matrix U = F_BB - F_BI X F_IB (still in the child's front,
// rows and columns [s_c, ns_c)) is added into the parent front at the rows and
// columns of the child map.
template <typename R>
__global__ void __launch_bounds__(256) nd_extend_kernel(NdKParams K, int slot) {
  using C = Cx<R>;
  const int f = K.list[blockIdx.y];
  const NdFront fr = K.fr[f];
  const int* nd = K.T.node + fr.node * kNdNodeInts;
  const int c = nd[slot ? ND_C1 : ND_C0];
  if (c < 0) return;
  const int fc = f - fr.node + c;  // the child front of the same slab
  const Slab Ec = K.eslab[fc], Ep = K.eslab[f];
  const int sc = Ec.np, Bc = Ec.nb - sc, w = fr.w;
  const int b = blockIdx.x;
  if (b >= Bc) return;
  const int* cm = K.T.cmap + K.T.node[c * kNdNodeInts + ND_OFFM];
  const int pr = cm[b / w] * w + (b % w);
  const C* src = reinterpret_cast<const C*>(K.A) + Ec.aoff + (long long)(sc + b) * Ec.ld + sc;
  C* dst = reinterpret_cast<C*>(K.A) + Ep.aoff + (long long)pr * Ep.ld;
  for (int j = threadIdx.x; j < Bc; j += blockDim.x) {
    const int pc = cm[j / w] * w + (j % w);
    dst[pc] = cadd(dst[pc], src[j]);
  }
}

// After the Gauss-Jordan steps on the I columns (pivot of column c in physical
// row piv_row[c], col_of_row its inverse on the I rows) the front holds, with
// i, c < s, j < B and b < B:
//   X[c][i]  = F[piv_row[c]][col_of_row[i]]
//   P[c][j]  = F[piv_row[c]][s + j]             (P = X F_IB)
//   L[b][i]  = -F[s + b][col_of_row[i]]         (L = F_BI X)
// Row r = blockIdx.x of [X; L] (and of P for r < s) of front list[blockIdx.y].
template <typename R>
__global__ void __launch_bounds__(256) nd_store_kernel(NdKParams K) {
  using C = Cx<R>;
  const int f = K.list[blockIdx.y];
  const Slab E = K.eslab[f];
  const int r = blockIdx.x;
  if (r >= E.nb) return;
  const NdFront fr = K.fr[f];
  const int s = E.np, B = E.nb - s, ld = E.ld;
  const int* piv_row = K.piv + E.poff;
  const int* col_of_row = piv_row + E.nb;
  const C* A = reinterpret_cast<const C*>(K.A) + E.aoff;
  C* XL = reinterpret_cast<C*>(K.W) + fr.xl + (long long)r * fr.lds;
  if (r < s) {
    const C* src = A + (long long)min(max(piv_row[r], 0), s - 1) * ld;
    for (int i = threadIdx.x; i < s; i += blockDim.x) XL[i] = src[min(max(col_of_row[i], 0), s - 1)];
    C* Pr = reinterpret_cast<C*>(K.W) + fr.pf + (long long)r * fr.ldb;
    for (int j = threadIdx.x; j < B; j += blockDim.x) Pr[j] = src[s + j];
  } else {
    const C* src = A + (long long)r * ld;
    for (int i = threadIdx.x; i < s; i += blockDim.x) {
      const C v = src[min(max(col_of_row[i], 0), s - 1)];
      XL[i] = cmake<R>(-v.x, -v.y);
    }
  }
}

// ------------------------------------------------------------ solves
constexpr int kNdSolveThreads = 256;
constexpr int kNdWarps = kNdSolveThreads / 32;
constexpr int kNdRowsPerWarp = 2;
constexpr int kNdRowsPerItem = kNdWarps * kNdRowsPerWarp;

struct NdSolveParams {
  NdTab T;
  const NdFront* fr;
  const Slab* eslab;
  const Slab* slabs;
  const Solve3Job* jobs;
  const int* nodes;   // node ids of this depth
  const void* W;
  void* x;            // natural-order slab vectors (per slab at Slab::zoff): input, then the solution
  void* zu;           // per-front scratch: z (s rows) then u (B rows)
  int ldv;
  // input and output of the batch (as the block-elimination solve)
  const void* in;
  void* outM;
  void* outR;
  void* outL;
  void* outSub;
  double inv_h2;
};

// natural slab-local index of unknown (column col, plane i3l): (i2*w + i3l)*n + i1
__device__ __forceinline__ long long nd_nat(int col, int i3l, int w, int n) {
  const int i1 = col % n, i2 = col / n;
  return ((long long)i2 * w + i3l) * n + i1;
}

// y[rr][q] = M[row_rr][0..len) . v[0..len)[q] for the warp's rows (lane-strided)
template <typename R, int NR>
__device__ __forceinline__ void nd_rows(const Cx<R>* M, long long ldm, int rowa, int nrows, int len,
                                        const Cx<R>* v, Cx<R> (&y)[kNdRowsPerWarp][NR]) {
  using C = Cx<R>;
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int rr = 0; rr < kNdRowsPerWarp; ++rr)
#pragma unroll
    for (int q = 0; q < NR; ++q) y[rr][q] = czero<R>();
  const C* m0 = M + (long long)min(rowa, nrows - 1) * ldm;
  const C* m1 = M + (long long)min(rowa + 1, nrows - 1) * ldm;
  for (int j = lane; j < len; j += 32) {
    const C a = m0[j], b = m1[j];
#pragma unroll
    for (int q = 0; q < NR; ++q) {
      const C vv = v[j * NR + q];
      cfma(y[0][q], a, vv);
      cfma(y[1][q], b, vv);
    }
  }
#pragma unroll
  for (int rr = 0; rr < kNdRowsPerWarp; ++rr)
#pragma unroll
    for (int q = 0; q < NR; ++q)
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        y[rr][q].x += __shfl_xor_sync(0xffffffffu, y[rr][q].x, off);
        y[rr][q].y += __shfl_xor_sync(0xffffffffu, y[rr][q].y, off);
      }
}

// Forward step of one depth.  Grid (row chunks, nodes of the depth, jobs).
template <typename R, int NR>
__global__ void __launch_bounds__(kNdSolveThreads) nd_fwd_kernel(NdSolveParams P) {
  using C = Cx<R>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* fv = reinterpret_cast<C*>(smem_raw);  // [ns][NR]
  const Solve3Job J = P.jobs[blockIdx.z];
  const int node = P.nodes[blockIdx.y];
  const int f = J.slab * P.T.nn + node;
  const Slab E = P.eslab[f];
  const int ns = E.nb, s = E.np;
  const int row0 = blockIdx.x * kNdRowsPerItem;
  if (row0 >= ns) return;
  const NdFront fr = P.fr[f];
  const Slab S = P.slabs[J.slab];
  const int w = S.w, n = P.T.n, ldv = P.ldv;
  const int* nd = P.T.node + node * kNdNodeInts;
  const int* cI = P.T.cols + nd[ND_OFFC];
  const C* x = reinterpret_cast<const C*>(P.x) + S.zoff;
  const C* zu = reinterpret_cast<const C*>(P.zu);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int e = tid; e < ns * NR; e += kNdSolveThreads) {
    const int r = e / NR, q = e - r * NR;
    C v = czero<R>();
    if (r < s && q < J.nr) {
      const int ci = r / w;
      v = x[nd_nat(cI[ci], r - ci * w, w, n) * ldv + J.rhs0 + q];
    }
    fv[e] = v;
  }
  __syncthreads();
#pragma unroll
  for (int slot = 0; slot < 2; ++slot) {
    const int c = nd[slot ? ND_C1 : ND_C0];
    if (c >= 0) {  // block-uniform
      const int fc = J.slab * P.T.nn + c;
      const Slab Ec = P.eslab[fc];
      const int sc = Ec.np, Bc = Ec.nb - sc;
      const C* u = zu + P.fr[fc].zu + (long long)sc * ldv;
      const int* cm = P.T.cmap + P.T.node[c * kNdNodeInts + ND_OFFM];
      for (int e = tid; e < Bc * NR; e += kNdSolveThreads) {
        const int b = e / NR, q = e - b * NR;
        if (q < J.nr) {
          const int pos = cm[b / w] * w + (b % w);
          fv[pos * NR + q] = cadd(fv[pos * NR + q], u[(long long)b * ldv + J.rhs0 + q]);
        }
      }
      __syncthreads();
    }
  }
  const int rowa = row0 + warp * kNdRowsPerWarp;
  if (rowa >= ns) return;
  C y[kNdRowsPerWarp][NR];
  nd_rows<R, NR>(reinterpret_cast<const C*>(P.W) + fr.xl, fr.lds, rowa, ns, s, fv, y);
  if (lane == 0) {
    C* out = reinterpret_cast<C*>(P.zu) + fr.zu;
#pragma unroll
    for (int rr = 0; rr < kNdRowsPerWarp; ++rr) {
      const int row = rowa + rr;
      if (row >= ns) break;
#pragma unroll
      for (int q = 0; q < NR; ++q) {
        if (q >= J.nr) continue;
        C v = y[rr][q];
        if (row >= s) v = csub(fv[row * NR + q], v);  // u = f_B - L f_I
        out[(long long)row * ldv + J.rhs0 + q] = v;   // z = X f_I
      }
    }
  }
}

// Backward step of one depth: x_I = z - P x_B.  Grid (row chunks, nodes, jobs).
template <typename R, int NR>
__global__ void __launch_bounds__(kNdSolveThreads) nd_bwd_kernel(NdSolveParams P) {
  using C = Cx<R>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* xb = reinterpret_cast<C*>(smem_raw);  // [B][NR]
  const Solve3Job J = P.jobs[blockIdx.z];
  const int node = P.nodes[blockIdx.y];
  const int f = J.slab * P.T.nn + node;
  const Slab E = P.eslab[f];
  const int s = E.np, B = E.nb - s;
  const int row0 = blockIdx.x * kNdRowsPerItem;
  if (row0 >= s) return;
  const NdFront fr = P.fr[f];
  const Slab S = P.slabs[J.slab];
  const int w = S.w, n = P.T.n, ldv = P.ldv;
  const int* nd = P.T.node + node * kNdNodeInts;
  const int ncI = nd[ND_NCI];
  const int* cI = P.T.cols + nd[ND_OFFC];
  const int* cB = cI + ncI;
  C* x = reinterpret_cast<C*>(P.x) + S.zoff;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int e = tid; e < B * NR; e += kNdSolveThreads) {
    const int b = e / NR, q = e - b * NR;
    C v = czero<R>();
    if (q < J.nr) {
      const int ci = b / w;
      v = x[nd_nat(cB[ci], b - ci * w, w, n) * ldv + J.rhs0 + q];
    }
    xb[e] = v;
  }
  __syncthreads();
  const int rowa = row0 + warp * kNdRowsPerWarp;
  if (rowa >= s) return;
  C y[kNdRowsPerWarp][NR];
  if (B > 0) {
    nd_rows<R, NR>(reinterpret_cast<const C*>(P.W) + fr.pf, fr.ldb, rowa, s, B, xb, y);
  } else {
#pragma unroll
    for (int rr = 0; rr < kNdRowsPerWarp; ++rr)
#pragma unroll
      for (int q = 0; q < NR; ++q) y[rr][q] = czero<R>();
  }
  if (lane == 0) {
    const C* z = reinterpret_cast<const C*>(P.zu) + fr.zu;
#pragma unroll
    for (int rr = 0; rr < kNdRowsPerWarp; ++rr) {
      const int row = rowa + rr;
      if (row >= s) break;
      const int ci = row / w;
      const long long nat = nd_nat(cI[ci], row - ci * w, w, n);
#pragma unroll
      for (int q = 0; q < NR; ++q) {
        if (q >= J.nr) continue;
        x[nat * ldv + J.rhs0 + q] = csub(z[(long long)row * ldv + J.rhs0 + q], y[rr][q]);
      }
    }
  }
}

// Right-hand side of every job into its slab's natural-order vector: the
// subproblem's g as Algorithm 2 forms it (see the block-elimination solve).
// Grid (chunks of the slab's unknowns, jobs).
template <typename R>
__global__ void __launch_bounds__(256) nd_input_kernel(NdSolveParams P) {
  using C = Cx<R>;
  const Solve3Job J = P.jobs[blockIdx.y];
  const Slab S = P.slabs[J.slab];
  const int n = P.T.n, nb = S.nb, ldv = P.ldv;
  const long long total = (long long)n * nb * J.nr;
  C* x = reinterpret_cast<C*>(P.x) + S.zoff;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long nat = e / J.nr;
    const int q = (int)(e - nat * J.nr);
    const int k = (int)(nat / nb), j = (int)(nat - (long long)k * nb);
    const int i3l = j / n, i1 = j - i3l * n;
    const int col = J.rhs0 + q;
    C v = czero<R>();
    if (J.mode == MODE_EMBED) {
      if (i3l >= S.xoff && i3l < S.xoff + S.xw)
        v = reinterpret_cast<const C*>(P.in)[((long long)((S.lo - 1 + i3l) * n + k) * n + i1) * ldv + col];
    } else if (J.mode == MODE_FILL_R || J.mode == MODE_FILL_L) {
      const bool edge = (J.mode == MODE_FILL_R) ? (i3l == 0) : (i3l == S.w - 1);
      if (edge) {
        const long long idx = ((long long)(S.src_plane * n + k) * n + i1) * ldv + col;
        v = reinterpret_cast<const C*>(P.outM)[idx];
        if (S.src_sweep)
          v = cadd(v, reinterpret_cast<const C*>(J.mode == MODE_FILL_R ? P.outR : P.outL)[idx]);
        v.x *= (R)(-P.inv_h2);
        v.y *= (R)(-P.inv_h2);
      }
    } else {  // MODE_SUB
      v = reinterpret_cast<const C*>(P.in)[((long long)(i3l * n + k) * n + i1) * ldv + col];
    }
    x[nat * ldv + col] = v;
  }
}

// The solution of every job from its natural-order vector into the outputs
// (restricted to X_p for the apply, whole for MODE_SUB).
template <typename R>
__global__ void __launch_bounds__(256) nd_output_kernel(NdSolveParams P) {
  using C = Cx<R>;
  const Solve3Job J = P.jobs[blockIdx.y];
  const Slab S = P.slabs[J.slab];
  const int n = P.T.n, nb = S.nb, ldv = P.ldv;
  const long long total = (long long)n * nb * J.nr;
  const C* x = reinterpret_cast<const C*>(P.x) + S.zoff;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long nat = e / J.nr;
    const int q = (int)(e - nat * J.nr);
    const int k = (int)(nat / nb), j = (int)(nat - (long long)k * nb);
    const int i3l = j / n, i1 = j - i3l * n;
    const int col = J.rhs0 + q;
    const C v = x[nat * ldv + col];
    if (J.mode == MODE_SUB) {
      reinterpret_cast<double2*>(P.outSub)[((long long)(i3l * n + k) * n + i1) * ldv + col] =
          make_double2((double)v.x, (double)v.y);
    } else if (i3l >= S.xoff && i3l < S.xoff + S.xw) {
      const long long idx = ((long long)((S.lo - 1 + i3l) * n + k) * n + i1) * ldv + col;
      C* out = reinterpret_cast<C*>(J.mode == MODE_EMBED ? P.outM : J.mode == MODE_FILL_R ? P.outR : P.outL);
      out[idx] = v;
    }
  }
}

}  // namespace

}  // namespace asp

namespace asp {

namespace {

NdTab tab_of(const Handle& H) {
  NdTab T;
  T.node = H.d_ndtab;
  T.cols = H.d_ndtab + (size_t)H.ndt.nn * kNdNodeInts;
  T.cmap = T.cols + H.ndt.cols.size();
  T.nn = H.ndt.nn;
  T.n = H.n;
  return T;
}

// Largest per-launch list: grid.y of the front kernels.
constexpr int kNdMaxList = 32768;

}  // namespace

// Plans the fronts of every slab, their factor, work, pivot and scratch
// offsets and the factor's launch levels, and allocates the device data.  The
// handle's slabs are set up; W, A3 and piv3 hold placeholders.
int nd_setup(Handle& H) {
  std::string why;
  if (!nd_build_tree(H.n, H.ndt, &why)) return fail(ASP_ERR_INVALID, why);
  const NdTree& T = H.ndt;
  const int nn = T.nn, D = T.maxdepth + 1;
  std::vector<int> widths, kinds;
  for (const Slab& S : H.slabs) {
    widths.push_back(S.w);
    kinds.push_back(S.kind);
  }
  const int esz = H.prec == ASP_PREC_C128 ? 16 : 8;
  const int mr = H.prm.max_rhs;
  std::vector<int> chunk;
  const NdSizes Z = nd_sizes(T, widths, kinds, mr, esz, &chunk);
  H.nd_maxfront = Z.max_front;
  // the solve stages a front's vector for 4 right-hand sides in shared memory
  if ((long long)Z.max_front * 4 * esz > 200 * 1024)
    return fail(ASP_ERR_UNSUPPORTED, "nested dissection: the largest front (" + std::to_string(Z.max_front) +
                                         " unknowns) does not fit the solve's shared-memory stage");
  const long long NF = (long long)H.slabs.size() * nn;
  H.ndf_host.assign(NF, NdFront{});
  std::vector<Slab> es(NF);
  long long xl = 0, poff = 0, zu = 0;
  for (size_t i = 0; i < H.slabs.size(); ++i) {
    const int w = widths[i];
    for (int t = 0; t < nn; ++t) {
      const long long f = (long long)i * nn + t;
      const int s = T.node[t * kNdNodeInts + ND_NCI] * w, B = T.node[t * kNdNodeInts + ND_NCB] * w;
      const int ns = s + B;
      NdFront& fr = H.ndf_host[f];
      fr.slab = (int)i;
      fr.node = t;
      fr.w = w;
      fr.lds = r4(s);
      fr.ldb = r4(B);
      fr.xl = xl;
      xl += (long long)ns * fr.lds;
      fr.pf = xl;
      xl += (long long)s * fr.ldb;
      fr.zu = zu;
      zu += (long long)ns * mr;
      Slab E = H.slabs[i];
      E.nb = ns;
      E.ld = r4(ns);
      E.np = s;
      E.zbo = (long long)ns * E.ld;
      E.poff = poff;
      poff += 3LL * ns;
      es[f] = E;
    }
  }
  // work offsets and launch levels: per group (0: M slabs, 1: R and L slabs),
  // per chunk, per depth (deepest first); fronts of even depths in the group's
  // first parity buffer, odd depths in the second
  std::vector<int> lists;
  H.nd_levels.clear();
  long long gbase = 0;
  for (int g = 0; g < 2; ++g) {
    int nck = 0;
    for (size_t i = 0; i < widths.size(); ++i)
      if ((kinds[i] == KIND_M) == (g == 0)) nck = std::max(nck, chunk[i] + 1);
    // sizes of each (chunk, depth) level
    std::vector<std::vector<long long>> lev(nck, std::vector<long long>(D, 0));
    for (size_t i = 0; i < widths.size(); ++i) {
      if ((kinds[i] == KIND_M) != (g == 0)) continue;
      for (int t = 0; t < nn; ++t)
        lev[chunk[i]][T.node[t * kNdNodeInts + ND_DEPTH]] += front_work(es[(long long)i * nn + t].nb);
    }
    long long buf[2] = {0, 0};
    for (int c = 0; c < nck; ++c)
      for (int d = 0; d < D; ++d) buf[d % 2] = std::max(buf[d % 2], lev[c][d]);
    for (int c = 0; c < nck; ++c) {
      for (int d = D - 1; d >= 0; --d) {
        long long off = gbase + (d % 2 ? buf[0] : 0);
        Handle::NdLevel L;
        L.off = (int)lists.size();
        L.depth = d;
        L.group = g;
        auto flush = [&]() {
          if (L.count > 0) H.nd_levels.push_back(L);
          L = Handle::NdLevel();
          L.off = (int)lists.size();
          L.depth = d;
          L.group = g;
        };
        for (size_t i = 0; i < widths.size(); ++i) {
          if ((kinds[i] == KIND_M) != (g == 0) || chunk[i] != c) continue;
          for (int t : T.at_depth[d]) {
            const long long f = (long long)i * nn + t;
            Slab& E = es[f];
            E.aoff = off;
            off += front_work(E.nb);
            if (L.count == kNdMaxList) flush();
            lists.push_back((int)f);
            L.count++;
            L.nbmax = std::max(L.nbmax, E.nb);
            L.npmax = std::max(L.npmax, E.np);
            for (int slot = 0; slot < 2; ++slot) {
              const int ch = T.node[t * kNdNodeInts + (slot ? ND_C1 : ND_C0)];
              if (ch >= 0) L.bmax = std::max(L.bmax, T.node[ch * kNdNodeInts + ND_NCB] * widths[i]);
            }
          }
        }
        flush();
      }
    }
    gbase += buf[0] + buf[1];
  }
  // complex64: the levels with large fronts get tensor-core update operands
  // (one area per factor group, shared by its levels, which run in order)
  std::vector<std::vector<long long>> tc_rowA;
  std::vector<long long> tc_rows;
  std::vector<int> tc_group;
  long long area_rows[2] = {0, 0};
  if (H.prec == ASP_PREC_C64) {
    for (auto& L : H.nd_levels) {
      if (L.nbmax < kNdTcMinFront) continue;
      std::vector<long long> ra;
      long long rows = 0;
      for (int e = 0; e < L.count; ++e) {
        ra.push_back(rows);
        rows += (es[lists[L.off + e]].nb + 127) / 128 * 128;
      }
      L.tc = (int)tc_rowA.size();
      tc_rowA.push_back(ra);
      tc_rows.push_back(rows);
      tc_group.push_back(L.group);
      area_rows[L.group] = std::max(area_rows[L.group], rows);
    }
  }
  // per-depth node lists and column maxima (the solve's grids)
  std::vector<int> tab(T.node.begin(), T.node.end());
  tab.insert(tab.end(), T.cols.begin(), T.cols.end());
  tab.insert(tab.end(), T.cmap.begin(), T.cmap.end());
  H.nd_dep_off.assign(D, 0);
  H.nd_dep_nc.assign(D, 0);
  H.nd_dep_nci.assign(D, 0);
  H.nd_dep_ncb.assign(D, 0);
  for (int d = 0; d < D; ++d) {
    H.nd_dep_off[d] = (int)tab.size();
    for (int t : T.at_depth[d]) {
      tab.push_back(t);
      H.nd_dep_nc[d] = std::max(H.nd_dep_nc[d], T.nc(t));
      H.nd_dep_nci[d] = std::max(H.nd_dep_nci[d], T.node[t * kNdNodeInts + ND_NCI]);
      H.nd_dep_ncb[d] = std::max(H.nd_dep_ncb[d], T.node[t * kNdNodeInts + ND_NCB]);
    }
  }
  // device data (the placeholders of W, A3 and piv3 are replaced)
  cudaFree(H.W);
  cudaFree(H.A3);
  cudaFree(H.piv3);
  H.W = nullptr;
  H.A3 = nullptr;
  H.piv3 = nullptr;
  H.W_elems = (size_t)xl;
  bool ok = true;
  auto dal = [&](void** p, size_t bytes) {
    if (ok && dev_malloc(p, bytes ? bytes : 16) != cudaSuccess) {
      ok = false;
      *p = nullptr;
    }
  };
  dal(&H.W, (size_t)xl * esz);
  dal(&H.A3, (size_t)gbase * esz);
  dal((void**)&H.piv3, (size_t)poff * sizeof(int));
  dal(&H.nd_zu, (size_t)zu * esz);
  dal((void**)&H.d_ndtab, tab.size() * sizeof(int));
  dal((void**)&H.d_ndf, H.ndf_host.size() * sizeof(NdFront));
  dal((void**)&H.d_ndslab, es.size() * sizeof(Slab));
  dal((void**)&H.d_ndlist, std::max<size_t>(lists.size(), 1) * sizeof(int));
  for (int g = 0; g < 2; ++g)
    if (area_rows[g] > 0) dal((void**)&H.nd_tc_area[g], (size_t)tc_group_floats(area_rows[g]) * sizeof(float));
  if (!ok) {
    cudaGetLastError();
    return fail(ASP_ERR_OOM, "nested dissection: device allocation failed");
  }
  auto up = [&](void* dst, const void* src, size_t bytes) {
    if (ok && bytes && cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice) != cudaSuccess) ok = false;
  };
  up(H.d_ndtab, tab.data(), tab.size() * sizeof(int));
  up(H.d_ndf, H.ndf_host.data(), H.ndf_host.size() * sizeof(NdFront));
  up(H.d_ndslab, es.data(), es.size() * sizeof(Slab));
  up(H.d_ndlist, lists.data(), lists.size() * sizeof(int));
  if (ok && cudaMemset(H.piv3, 0, (size_t)poff * sizeof(int)) != cudaSuccess) ok = false;
  if (ok && cudaMemset(H.W, 0, (size_t)xl * esz) != cudaSuccess) ok = false;
  if (!ok) return fail(ASP_ERR_CUDA, "nested dissection: uploading the plan");
  H.nd_tcg.assign(tc_rowA.size(), TcGroup());
  for (size_t i = 0; i < tc_rowA.size(); ++i) {
    const int rc = tc_group_setup(H.nd_tcg[i], H.nd_tc_area[tc_group[i]], tc_rowA[i], tc_rows[i]);
    if (rc != ASP_OK) return rc;
  }
  return ASP_OK;
}

void nd_release(Handle& H) {
  if (H.d_ndtab) cudaFree(H.d_ndtab);
  if (H.d_ndf) cudaFree(H.d_ndf);
  if (H.d_ndslab) cudaFree(H.d_ndslab);
  if (H.d_ndlist) cudaFree(H.d_ndlist);
  if (H.nd_zu) cudaFree(H.nd_zu);
  for (auto& g : H.nd_tcg) tc_group_release(g);
  H.nd_tcg.clear();
  for (int g = 0; g < 2; ++g) {
    if (H.nd_tc_area[g]) cudaFree(H.nd_tc_area[g]);
    H.nd_tc_area[g] = nullptr;
  }
  H.d_ndtab = nullptr;
  H.d_ndf = nullptr;
  H.d_ndslab = nullptr;
  H.d_ndlist = nullptr;
  H.nd_zu = nullptr;
}

namespace {

template <typename R> cudaError_t nd_level(Handle& H, const Handle::NdLevel& L, const FactorCoefs<R>& F,
                                           cudaStream_t s) {
  NdKParams K{};
  K.T = tab_of(H);
  K.fr = H.d_ndf;
  K.eslab = H.d_ndslab;
  K.slabs = H.d_slabs;
  K.list = H.d_ndlist + L.off;
  K.A = H.A3;
  K.piv = H.piv3;
  K.W = H.W;
  nd_assemble_kernel<R><<<dim3(L.nbmax, L.count), 256, 0, s>>>(K, F);
  H.launches += 1;
  if (L.bmax > 0) {
    nd_extend_kernel<R><<<dim3(L.bmax, L.count), 256, 0, s>>>(K, 0);
    nd_extend_kernel<R><<<dim3(L.bmax, L.count), 256, 0, s>>>(K, 1);
    H.launches += 2;
  }
  Slab3Params P{};
  P.slabs = H.d_ndslab;
  P.list = H.d_ndlist + L.off;
  P.nlist = L.count;
  P.n = H.n;
  P.W = H.W;
  P.A = H.A3;
  P.piv = H.piv3;
  P.err = H.err;
  const TcGroup* tc = L.tc >= 0 ? &H.nd_tcg[L.tc] : nullptr;  // complex64 large fronts: tensor cores
  cudaError_t e = gj_partial(H, P, L.nbmax, L.npmax, tc, s);
  if (e != cudaSuccess) return e;
  nd_store_kernel<R><<<dim3(L.nbmax, L.count), 256, 0, s>>>(K);
  H.launches += 1;
  return cudaGetLastError();
}

template <typename R> cudaError_t nd_factor_t(Handle& H, const FactorCoefs<R>& F, cudaStream_t s) {
  // the two groups' levels are enqueued alternately on their own streams
  std::vector<const Handle::NdLevel*> per[2];
  for (const auto& L : H.nd_levels) per[L.group].push_back(&L);
  cudaStream_t gs[2];
  for (int g = 0; g < 2; ++g) {
    gs[g] = s;
    if (g < (int)H.fgroups.size() && H.fgroups[g].stream) gs[g] = H.fgroups[g].stream;
  }
  PhaseTok tk[2];
  for (int g = 0; g < 2; ++g) tk[g] = phase_begin(H, PH_FACTOR, gs[g]);
  cudaError_t e = cudaSuccess;
  const size_t nmax = std::max(per[0].size(), per[1].size());
  for (size_t k = 0; k < nmax && e == cudaSuccess; ++k)
    for (int g = 0; g < 2 && e == cudaSuccess; ++g)
      if (k < per[g].size()) e = nd_level<R>(H, *per[g][k], F, gs[g]);
  for (int g = 0; g < 2; ++g) phase_end(H, tk[g], gs[g]);
  return e;
}

}  // namespace

int nd_factor(Handle& H, cudaStream_t s) {
  auto cuda_fail = [](const char* what, cudaError_t e) {
    return fail(ASP_ERR_CUDA, std::string("3D nested-dissection factor: ") + what + ": " + cudaGetErrorString(e));
  };
  cudaError_t e = cudaEventRecord(H.ev_fork, s);
  if (e != cudaSuccess) return cuda_fail("fork record", e);
  for (auto& g : H.fgroups)
    if (g.stream && (e = cudaStreamWaitEvent(g.stream, H.ev_fork, 0)) != cudaSuccess) return cuda_fail("fork wait", e);
  const cudaError_t launch_err =
      H.prec == ASP_PREC_C128 ? nd_factor_t<double>(H, H.fc64, s) : nd_factor_t<float>(H, H.fc32, s);
  for (auto& g : H.fgroups) {
    if (!g.stream) continue;
    if ((e = cudaEventRecord(g.done, g.stream)) != cudaSuccess) return cuda_fail("join record", e);
    if ((e = cudaStreamWaitEvent(s, g.done, 0)) != cudaSuccess) return cuda_fail("join wait", e);
  }
  if (launch_err != cudaSuccess) return cuda_fail("launch", launch_err);
  return ASP_OK;
}

namespace {

template <typename R, int NR>
cudaError_t nd_solve_t(Handle& H, const Solve3Params& Q, int nbmax, cudaStream_t s) {
  using C = Cx<R>;
  NdSolveParams P{};
  P.T = tab_of(H);
  P.fr = H.d_ndf;
  P.eslab = H.d_ndslab;
  P.slabs = H.d_slabs;
  P.jobs = Q.jobs;
  P.W = H.W;
  P.x = H.z3;
  P.zu = H.nd_zu;
  P.ldv = Q.ldv;
  P.in = Q.in;
  P.outM = Q.outM;
  P.outR = Q.outR;
  P.outL = Q.outL;
  P.outSub = Q.outSub;
  P.inv_h2 = Q.inv_h2;
  const int njobs = Q.njobs;
  if (njobs <= 0) return cudaSuccess;
  const int wmax = std::max(1, nbmax / std::max(H.n, 1));
  const int D = H.ndt.maxdepth + 1;
  const long long slab_elems = (long long)H.n * nbmax * NR;
  const int vgrid = (int)std::max<long long>(1, std::min<long long>((slab_elems + 255) / 256, 4LL * H.num_sms));
  nd_input_kernel<R><<<dim3(vgrid, njobs), 256, 0, s>>>(P);
  H.launches += 1;
  size_t smax = 0;
  for (int d = 0; d < D; ++d) smax = std::max(smax, (size_t)H.nd_dep_nc[d] * wmax * NR * sizeof(C));
  cudaError_t e = ensure_dyn_smem((const void*)nd_fwd_kernel<R, NR>, smax);
  if (e != cudaSuccess) return e;
  if ((e = ensure_dyn_smem((const void*)nd_bwd_kernel<R, NR>, smax)) != cudaSuccess) return e;
  for (int d = D - 1; d >= 0; --d) {
    P.nodes = H.d_ndtab + H.nd_dep_off[d];
    const int nodes = (int)H.ndt.at_depth[d].size();
    const int rows = H.nd_dep_nc[d] * wmax;
    const size_t sm = (size_t)rows * NR * sizeof(C);
    nd_fwd_kernel<R, NR><<<dim3((rows + kNdRowsPerItem - 1) / kNdRowsPerItem, nodes, njobs), kNdSolveThreads, sm,
                           s>>>(P);
    H.launches += 1;
  }
  for (int d = 0; d < D; ++d) {
    P.nodes = H.d_ndtab + H.nd_dep_off[d];
    const int nodes = (int)H.ndt.at_depth[d].size();
    const int rows = H.nd_dep_nci[d] * wmax;
    const size_t sm = (size_t)std::max(1, H.nd_dep_ncb[d] * wmax) * NR * sizeof(C);
    nd_bwd_kernel<R, NR><<<dim3((rows + kNdRowsPerItem - 1) / kNdRowsPerItem, nodes, njobs), kNdSolveThreads, sm,
                           s>>>(P);
    H.launches += 1;
  }
  nd_output_kernel<R><<<dim3(vgrid, njobs), 256, 0, s>>>(P);
  H.launches += 1;
  return cudaGetLastError();
}

}  // namespace

cudaError_t nd_solve(Handle& H, const Solve3Params& P, int NR, int nbmax, cudaStream_t s) {
  if (H.prec == ASP_PREC_C128) {
    if (NR == 4) return nd_solve_t<double, 4>(H, P, nbmax, s);
    if (NR == 2) return nd_solve_t<double, 2>(H, P, nbmax, s);
    return nd_solve_t<double, 1>(H, P, nbmax, s);
  }
  if (NR == 4) return nd_solve_t<float, 4>(H, P, nbmax, s);
  if (NR == 2) return nd_solve_t<float, 2>(H, P, nbmax, s);
  return nd_solve_t<float, 1>(H, P, nbmax, s);
}

}  // namespace asp
