// IJK-partitioned multi-process planning (Sec. III.A.1-III.A.3), host code only.
//
// Ownership: individual stored blocks (i <= j <= k) of compact T3/R3, balanced by a
// per-block cost with the longest-processing-time-first rule.  Exchange: the
// step (v) contractions of Sec. III.A.2 read T3 blocks owned elsewhere; the blocks
// are gathered in batches that partition them (each element sent once per cycle),
// consecutive in storage order and cut at equal shares of the step (v) work.  The
// work a gathered block causes on a rank follows the reads of the residual terms
// with unpacking of every block that rank owns:
//   F_oo:   3 positions x o values of l, block (l, i2, i3)            v^3 each
//   W_oooo: 3 pairs x o^2 values of (l, m), block (l, m, i3)          v^3 each
//   rings:  3 positions x o values of l, blocks (l, i2, i3), (i2, l, i3),
//           (i3, l, i2); 6 orderings x o values of l, block (i2, l, i3) v^4 each
// where (i1, i2, i3) runs over the orderings of the block's occupied labels each
// term takes.
#include <algorithm>
#include <cmath>
#include <new>
#include <numeric>
#include <vector>

#include "rccsdt.h"

namespace {

inline long long binom3(long long n) { return n < 3 ? 0 : n * (n - 1) * (n - 2) / 6; }
inline long long binom2(long long n) { return n < 2 ? 0 : n * (n - 1) / 2; }

// Storage index of the sorted triple (i <= j <= k): C(k+2,3) + C(j+1,2) + i.
inline int blk_sorted(int a, int b, int c) {
  if (a > b) std::swap(a, b);
  if (b > c) std::swap(b, c);
  if (a > b) std::swap(a, b);
  return (int)(binom3(c + 2) + binom2(b + 1) + a);
}

struct Triple {
  int i, j, k;
};

std::vector<Triple> triples(int o) {
  std::vector<Triple> t((size_t)o * (o + 1) * (o + 2) / 6);
  for (int k = 0; k < o; ++k)
    for (int j = 0; j <= k; ++j)
      for (int i = 0; i <= j; ++i) t[(size_t)blk_sorted(i, j, k)] = {i, j, k};
  return t;
}

// Calls f(u, fma) for every step (v) read of block t's residual terms.
template <class F>
void for_each_read(const Triple& t, int o, double v3, double v4, F&& f) {
  const int x[3] = {t.i, t.j, t.k};
  // F_oo: the position p of l's label, the other two stay
  for (int p = 0; p < 3; ++p) {
    const int i2 = x[p == 0 ? 1 : 0], i3 = x[p == 2 ? 1 : 2];
    for (int l = 0; l < o; ++l) f(blk_sorted(l, i2, i3), v3);
  }
  // W_oooo: the pair (p, q) replaced by (l, m), the third label stays
  for (int p = 0; p < 3; ++p) {
    const int i3 = x[p];
    for (int l = 0; l < o; ++l)
      for (int m = 0; m < o; ++m) f(blk_sorted(l, m, i3), v3);
  }
  // rings with the output's first label at position p: three reads per l
  for (int p = 0; p < 3; ++p) {
    const int i2 = x[p == 0 ? 1 : 0], i3 = x[p == 2 ? 1 : 2];
    for (int l = 0; l < o; ++l) {
      f(blk_sorted(l, i2, i3), v4);
      f(blk_sorted(i2, l, i3), v4);
      f(blk_sorted(i3, l, i2), v4);
    }
  }
  // ring over all six orderings (i1, i2, i3): block (i2, l, i3)
  static const int perm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  for (const auto& pm : perm)
    for (int l = 0; l < o; ++l) f(blk_sorted(x[pm[1]], l, x[pm[2]]), v4);
}

}  // namespace

struct rccsdt_ijk_plan {
  int o = 0, v = 0, nranks = 0, nbatches = 0;
  std::vector<double> cost;                 // [n3]
  std::vector<int> owner;                   // [n3]
  std::vector<std::vector<int>> local;      // per rank, storage order
  std::vector<int> cut;                     // batch b = blocks [cut[b], cut[b+1])
  std::vector<std::vector<int>> bcount;     // [batch][rank]
  std::vector<std::vector<int>> bblocks;    // [batch] grouped by owner
  std::vector<double> rank_cost;            // [nranks]
  std::vector<double> batch_work;           // [nbatches][nranks]
};

extern "C" int rccsdt_ijk_block_costs(int o, int v, double* cost) {
  if (o < 1 || v < 1 || o > 64 || !cost) return RCCSDT_ERR_ARG;
  const double V = v, O = o;
  const double full = 3.0 * V * V * V * V * V + 15.0 * O * V * V * V * V + 9.0 * V * V * V * V +
                      3.0 * O * O * V * V * V + 9.0 * O * V * V * V;
  const std::vector<Triple> t = triples(o);
  for (size_t b = 0; b < t.size(); ++b) cost[b] = (t[b].i == t[b].k) ? 0.0 : full;
  return RCCSDT_OK;
}

extern "C" int rccsdt_ijk_plan_create(int o, int v, int nranks, int batch_triples, const double* cost,
                                      rccsdt_ijk_plan** out) {
  if (!out) return RCCSDT_ERR_ARG;
  *out = nullptr;
  if (o < 1 || o > 64 || v < 1 || nranks < 1 || nranks > 4096 || batch_triples < 1) return RCCSDT_ERR_ARG;
  {
    const long long n3 = (long long)o * (o + 1) * (o + 2) / 6;
    const long long nb = std::min(n3, (n3 + batch_triples - 1) / batch_triples);
    if (nb * nranks > (1LL << 27)) return RCCSDT_ERR_ARG;  // the per-batch, per-rank work table
  }
  rccsdt_ijk_plan* p = new (std::nothrow) rccsdt_ijk_plan;
  if (!p) return RCCSDT_ERR_OOM;
  const std::vector<Triple> tr = triples(o);
  const int n3 = (int)tr.size();
  p->o = o;
  p->v = v;
  p->nranks = nranks;
  p->cost.resize((size_t)n3);
  if (cost) {
    for (int b = 0; b < n3; ++b) {
      if (!(cost[b] >= 0.0) || !std::isfinite(cost[b])) {
        delete p;
        return RCCSDT_ERR_ARG;
      }
      p->cost[(size_t)b] = cost[b];
    }
  } else {
    rccsdt_ijk_block_costs(o, v, p->cost.data());
  }

  // ownership: longest processing time first
  std::vector<int> order((size_t)n3);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return p->cost[(size_t)a] > p->cost[(size_t)b]; });
  p->owner.assign((size_t)n3, 0);
  p->rank_cost.assign((size_t)nranks, 0.0);
  std::vector<long long> nown((size_t)nranks, 0);
  for (int b : order) {
    int best = 0;
    for (int r = 1; r < nranks; ++r) {
      const double lr = p->rank_cost[(size_t)r], lb = p->rank_cost[(size_t)best];
      // equal load: fewer blocks first, so that zero-cost blocks spread too
      if (lr < lb || (lr == lb && nown[(size_t)r] < nown[(size_t)best])) best = r;
    }
    p->owner[(size_t)b] = best;
    p->rank_cost[(size_t)best] += p->cost[(size_t)b];
    ++nown[(size_t)best];
  }
  p->local.assign((size_t)nranks, {});
  for (int b = 0; b < n3; ++b) p->local[(size_t)p->owner[(size_t)b]].push_back(b);

  // step (v) work per gathered block, summed over readers
  const double v3 = (double)v * v * v, v4 = v3 * v;
  std::vector<double> tot((size_t)n3, 0.0);
  for (int t = 0; t < n3; ++t)
    if (p->cost[(size_t)t] > 0.0) for_each_read(tr[(size_t)t], o, v3, v4, [&](int u, double w) { tot[(size_t)u] += w; });

  // batches: consecutive blocks, cut at equal shares of the work (by count when no
  // block reads anything); every batch non-empty
  const int nb = std::min(n3, (n3 + batch_triples - 1) / batch_triples);
  p->nbatches = nb;
  std::vector<double> cum((size_t)n3 + 1, 0.0);
  for (int b = 0; b < n3; ++b) cum[(size_t)b + 1] = cum[(size_t)b] + tot[(size_t)b];
  const double total = cum[(size_t)n3];
  p->cut.assign((size_t)nb + 1, 0);
  p->cut[(size_t)nb] = n3;
  for (int q = 1; q < nb; ++q) {
    int c;
    if (total > 0.0) {
      const double target = total * q / nb;
      c = (int)(std::lower_bound(cum.begin(), cum.end(), target) - cum.begin());
    } else {
      c = (int)((long long)n3 * q / nb);
    }
    c = std::max(c, p->cut[(size_t)q - 1] + 1);
    c = std::min(c, n3 - (nb - q));
    p->cut[(size_t)q] = c;
  }
  std::vector<int> batch_of((size_t)n3);
  p->bcount.assign((size_t)nb, std::vector<int>((size_t)nranks, 0));
  p->bblocks.assign((size_t)nb, {});
  for (int q = 0; q < nb; ++q) {
    std::vector<int>& bl = p->bblocks[(size_t)q];
    for (int b = p->cut[(size_t)q]; b < p->cut[(size_t)q + 1]; ++b) {
      batch_of[(size_t)b] = q;
      ++p->bcount[(size_t)q][(size_t)p->owner[(size_t)b]];
      bl.push_back(b);
    }
    std::stable_sort(bl.begin(), bl.end(),
                     [&](int a, int b) { return p->owner[(size_t)a] < p->owner[(size_t)b]; });
  }
  p->batch_work.assign((size_t)nb * nranks, 0.0);
  for (int t = 0; t < n3; ++t) {
    if (!(p->cost[(size_t)t] > 0.0)) continue;
    const int r = p->owner[(size_t)t];
    for_each_read(tr[(size_t)t], o, v3, v4,
                  [&](int u, double w) { p->batch_work[(size_t)batch_of[(size_t)u] * nranks + r] += w; });
  }
  *out = p;
  return RCCSDT_OK;
}

extern "C" void rccsdt_ijk_plan_destroy(rccsdt_ijk_plan* plan) { delete plan; }

extern "C" int rccsdt_ijk_plan_info(const rccsdt_ijk_plan* p, long long info[6]) {
  if (!p || !info) return RCCSDT_ERR_ARG;
  long long own = 0, bmax = 0, smax = 0;
  for (const auto& l : p->local) own = std::max(own, (long long)l.size());
  for (int q = 0; q < p->nbatches; ++q) {
    bmax = std::max(bmax, (long long)p->bblocks[(size_t)q].size());
    for (int c : p->bcount[(size_t)q]) smax = std::max(smax, (long long)c);
  }
  info[0] = (long long)p->owner.size();
  info[1] = p->nranks;
  info[2] = p->nbatches;
  info[3] = own;
  info[4] = bmax;
  info[5] = smax;
  return RCCSDT_OK;
}

extern "C" int rccsdt_ijk_plan_owners(const rccsdt_ijk_plan* p, int* owner) {
  if (!p || !owner) return RCCSDT_ERR_ARG;
  std::copy(p->owner.begin(), p->owner.end(), owner);
  return RCCSDT_OK;
}

extern "C" int rccsdt_ijk_plan_local(const rccsdt_ijk_plan* p, int rank, int* blocks, int* count) {
  if (!p || !count || rank < 0 || rank >= p->nranks) return RCCSDT_ERR_ARG;
  const std::vector<int>& l = p->local[(size_t)rank];
  *count = (int)l.size();
  if (blocks) std::copy(l.begin(), l.end(), blocks);
  return RCCSDT_OK;
}

extern "C" int rccsdt_ijk_plan_batch(const rccsdt_ijk_plan* p, int b, int* counts, int* blocks) {
  if (!p || !counts || b < 0 || b >= p->nbatches) return RCCSDT_ERR_ARG;
  std::copy(p->bcount[(size_t)b].begin(), p->bcount[(size_t)b].end(), counts);
  if (blocks) std::copy(p->bblocks[(size_t)b].begin(), p->bblocks[(size_t)b].end(), blocks);
  return RCCSDT_OK;
}

extern "C" int rccsdt_ijk_plan_work(const rccsdt_ijk_plan* p, double* rank_cost, double* batch_work) {
  if (!p) return RCCSDT_ERR_ARG;
  if (rank_cost) std::copy(p->rank_cost.begin(), p->rank_cost.end(), rank_cost);
  if (batch_work) std::copy(p->batch_work.begin(), p->batch_work.end(), batch_work);
  return RCCSDT_OK;
}
