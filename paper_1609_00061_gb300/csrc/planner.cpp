// Host-side planning for the pixel array engine: polynomial bookkeeping, the
// valid tolerance of Sec. 3.2, the join order of Sec. 3.5 and cluster-tree
// costs.  Built with -ffp-contract=off so every double operation rounds once.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "pa_internal.h"
#include "planner.h"

namespace pa {

int64_t coeff_count(int n, int degree) {
  // C(n + degree, degree)
  int64_t r = 1;
  for (int i = 1; i <= degree; ++i) r = r * (n + i) / i;
  return r;
}

// Every exponent tuple of n variables with total degree <= degree, in graded
// lex order (degree ascending, then descending lexicographic).
static void graded_lex(int n, int degree, std::vector<std::vector<int>>& out) {
  out.clear();
  std::vector<int> e(n, 0);
  // recursive fill of position i with the remaining sum, largest value first
  struct Rec {
    static void go(int i, int n, int left, std::vector<int>& e, std::vector<std::vector<int>>& out) {
      if (i == n - 1) {
        e[i] = left;
        out.push_back(e);
        return;
      }
      for (int v = left; v >= 0; --v) {
        e[i] = v;
        go(i + 1, n, left - v, e, out);
      }
    }
  };
  for (int t = 0; t <= degree; ++t) {
    if (n == 0) {
      if (t == 0) out.push_back(e);
      continue;
    }
    Rec::go(0, n, t, e, out);
  }
}

static int64_t tuple_key(const std::vector<int>& e, int degree) {
  int64_t k = 0;
  for (int v : e) k = k * (degree + 1) + v;
  return k;
}

std::vector<int64_t> nest_order(int n, int degree) {
  std::vector<std::vector<int>> gl;
  graded_lex(n, degree, gl);
  // rank lookup by key
  std::vector<std::pair<int64_t, int64_t>> keyrank;
  keyrank.reserve(gl.size());
  for (size_t i = 0; i < gl.size(); ++i) keyrank.push_back({tuple_key(gl[i], degree), (int64_t)i});
  std::sort(keyrank.begin(), keyrank.end());
  std::vector<int64_t> order;
  order.reserve(gl.size());
  std::vector<int> e(n, 0);
  // visit(k, rem): the last variable outermost, each exponent ascending
  struct Visit {
    static void go(int k, int rem, int degree, std::vector<int>& e,
                   const std::vector<std::pair<int64_t, int64_t>>& kr, std::vector<int64_t>& order) {
      if (k < 0) {
        int64_t key = tuple_key(e, degree);
        auto it = std::lower_bound(kr.begin(), kr.end(), std::make_pair(key, (int64_t)-1));
        order.push_back(it->second);
        return;
      }
      for (int v = 0; v <= rem; ++v) {
        e[k] = v;
        go(k - 1, rem - v, degree, e, kr, order);
      }
      e[k] = 0;
    }
  };
  Visit::go(n - 1, degree, degree, e, keyrank, order);
  return order;
}

double valid_tolerance(int n, int degree, const double* coeffs, const double* lo,
                       const double* hi, const int32_t* res, double width) {
  std::vector<std::vector<int>> gl;
  graded_lex(n, degree, gl);
  double M[kMaxDim];
  for (int q = 0; q < n; ++q) M[q] = fmax(fabs(lo[q]), fabs(hi[q]));
  double total = 0.0;
  for (int p = 0; p < n; ++p) {
    double S = 0.0;
    for (size_t m = 0; m < gl.size(); ++m) {
      const std::vector<int>& e = gl[m];
      if (e[p] == 0) continue;
      double t = fabs(coeffs[m]) * (double)e[p];
      double pp = 1.0;
      for (int k = 1; k < e[p]; ++k) pp = pp * M[p];
      t = t * pp;
      for (int q = 0; q < n; ++q) {
        if (q == p) continue;
        double pq = 1.0;
        for (int k = 0; k < e[q]; ++k) pq = pq * M[q];
        t = t * pq;
      }
      S = S + t;
    }
    double delta = (hi[p] - lo[p]) / (double)res[p];
    total = total + S * (delta * width);
  }
  return total * (1.0 + 0x1p-30);
}

// ------------------------------------------------------------- join order
static double set_size(const std::vector<int>& vars, const std::vector<double>& vres) {
  double s = 1.0;
  for (int v : vars) s *= vres[v];
  return s;
}

static std::vector<int> set_union(const std::vector<int>& a, const std::vector<int>& b) {
  std::vector<int> u = a;
  for (int v : b)
    if (std::find(u.begin(), u.end(), v) == u.end()) u.push_back(v);
  return u;
}

Plan plan_joins(int nvars, const std::vector<double>& vres,
                const std::vector<std::vector<int>>& rel_vars, const std::vector<int>& exposed,
                int order, const int32_t* given_pairs) {
  return plan_joins_policy(nvars, vres, rel_vars, exposed, order, given_pairs, 0);
}

// ----------------------------------------------------- optimal cluster tree
// The pairwise cluster tree of least naive cost (Sec. 3.5: the cost of a tree
// is the sum over its clusters of r^Lambda, Lambda the links of the cluster's
// children; the parallel cost adds only the most expensive child chain).
// Dynamic programming over subsets S of a set of relations: S's result keeps
// K(S) = (variables of S) & (variables needed outside S), which does not
// depend on how S was joined, so
//   best(S) = min over splits S = S1 + S2 of best(S1) + best(S2) + r^(V(S1) | V(S2)),
// V(single relation) = its variables, V(S) = K(S) otherwise.  Ties go to the
// smaller parallel cost, then to the first split in enumeration order.  The
// search visits every pair (S, S1), about 3^n of them.
namespace {

struct TreeNode {
  int leaf = -1;     // relation index, or -1 for a join
  int left = -1, right = -1;
};

// Exact search over the relations `rels` (at most 20), whose results must
// keep every variable of `outside`.  Appends the optimal tree's nodes to
// `nodes` and returns the root node's index.
int exact_tree(const std::vector<int>& rels, const std::vector<uint64_t>& rmask, uint64_t outside,
               const std::vector<double>& vres, std::vector<TreeNode>& nodes) {
  const int n = (int)rels.size();
  auto size_of = [&](uint64_t m) {
    double s = 1.0;
    for (; m; m &= m - 1) s *= vres[__builtin_ctzll(m)];
    return s;
  };
  const uint32_t full = (1u << n) - 1;
  const size_t N = (size_t)1 << n;
  std::vector<double> cost(N, INFINITY), pcost(N, INFINITY);
  std::vector<uint64_t> vmask(N, 0), inner(N, 0);
  std::vector<uint32_t> split(N, 0);
  for (uint32_t S = 1; S <= full; ++S) {
    const uint32_t low = S & (~S + 1);
    inner[S] = inner[S & (S - 1)] | rmask[rels[__builtin_ctz(S)]];
    if (S == low) {
      cost[S] = pcost[S] = 0.0;
      vmask[S] = inner[S];
      continue;
    }
    uint64_t need = outside;
    for (uint32_t o = full & ~S; o; o &= o - 1) need |= rmask[rels[__builtin_ctz(o)]];
    vmask[S] = inner[S] & need;
    const double floor_node = size_of(vmask[S]);  // the root of S keeps at least K(S)
    // S1 runs over the proper submasks of S that hold S's lowest relation
    const uint32_t rest = S ^ low;
    for (uint32_t sub = (rest - 1) & rest;; sub = (sub - 1) & rest) {
      const uint32_t S1 = sub | low, S2 = S ^ S1;
      const double below = cost[S1] + cost[S2];
      if (below + floor_node <= cost[S]) {
        const double node = size_of(vmask[S1] | vmask[S2]);
        const double c = below + node;
        const double pc = node + std::max(pcost[S1], pcost[S2]);
        if (c < cost[S] || (c == cost[S] && pc < pcost[S])) {
          cost[S] = c;
          pcost[S] = pc;
          split[S] = S1;
        }
      }
      if (sub == 0) break;
    }
  }
  struct Emit {
    const std::vector<int>& rels;
    const std::vector<uint32_t>& split;
    std::vector<TreeNode>& nodes;
    int go(uint32_t S) {
      TreeNode t;
      if ((S & (S - 1)) == 0) {
        t.leaf = rels[__builtin_ctz(S)];
      } else {
        t.left = go(split[S]);
        t.right = go(S ^ split[S]);
      }
      nodes.push_back(t);
      return (int)nodes.size() - 1;
    }
  } emit{rels, split, nodes};
  return emit.go(full);
}

void tree_leaves(const std::vector<TreeNode>& nodes, int t, std::vector<int>& out) {
  if (nodes[t].leaf >= 0) {
    out.push_back(nodes[t].leaf);
    return;
  }
  tree_leaves(nodes, nodes[t].left, out);
  tree_leaves(nodes, nodes[t].right, out);
}

// Emit the joins of a tree bottom-up into a Plan (slots 0..nrel-1 are the
// relations; join t creates slot nrel + t).
int emit_plan(const std::vector<TreeNode>& nodes, int t, int nrel,
              const std::vector<std::vector<int>>& rel_vars, const std::vector<uint64_t>& rmask,
              uint64_t emask, const std::vector<double>& vres,
              std::vector<std::vector<int>>& slot_vars, Plan& out) {
  if (nodes[t].leaf >= 0) return nodes[t].leaf;
  const int a = emit_plan(nodes, nodes[t].left, nrel, rel_vars, rmask, emask, vres, slot_vars, out);
  const int b = emit_plan(nodes, nodes[t].right, nrel, rel_vars, rmask, emask, vres, slot_vars, out);
  std::vector<int> in;
  tree_leaves(nodes, t, in);
  uint64_t need = emask;
  for (int i = 0; i < nrel; ++i)
    if (std::find(in.begin(), in.end(), i) == in.end()) need |= rmask[i];
  Join jn;
  jn.a = a;
  jn.b = b;
  const std::vector<int> u = set_union(slot_vars[a], slot_vars[b]);
  for (int v : u)
    if (need >> v & 1) jn.keep.push_back(v);
  jn.cost = set_size(u, vres);
  out.joins.push_back(jn);
  out.pixel_ops += jn.cost;
  out.peak_bits = std::max(out.peak_bits, set_size(jn.keep, vres));
  slot_vars.push_back(jn.keep);
  return nrel + (int)out.joins.size() - 1;
}

}  // namespace

bool plan_optimal(int nvars, const std::vector<double>& vres,
                  const std::vector<std::vector<int>>& rel_vars, const std::vector<int>& exposed,
                  Plan& plan) {
  const int n = (int)rel_vars.size();
  if (n < 1 || nvars > 64) return false;
  std::vector<uint64_t> rmask(n, 0);
  for (int i = 0; i < n; ++i)
    for (int v : rel_vars[i]) rmask[i] |= 1ull << v;
  uint64_t emask = 0;
  for (int v : exposed) emask |= 1ull << v;
  std::vector<TreeNode> nodes;
  int root;
  if (n <= kMaxOptimalRelations) {
    std::vector<int> all(n);
    for (int i = 0; i < n; ++i) all[i] = i;
    root = exact_tree(all, rmask, emask, vres, nodes);
  } else {
    // larger networks: the greedy tree, every subtree of at most
    // kMaxOptimalRelations relations replaced by the exact optimum over its
    // relations (a subtree's result does not depend on its inner order)
    Plan g = plan_joins_policy(nvars, vres, rel_vars, exposed, PA_ORDER_GREEDY, nullptr, 0);
    std::vector<int> slot_node(n + g.joins.size());
    std::vector<std::vector<int>> slot_rels(n + g.joins.size());
    for (int i = 0; i < n; ++i) {
      TreeNode t;
      t.leaf = i;
      nodes.push_back(t);
      slot_node[i] = i;
      slot_rels[i] = {i};
    }
    std::vector<char> replaced(n + g.joins.size(), 0);
    for (size_t t = 0; t < g.joins.size(); ++t) {
      const int s = n + (int)t;
      slot_rels[s] = slot_rels[g.joins[t].a];
      slot_rels[s].insert(slot_rels[s].end(), slot_rels[g.joins[t].b].begin(),
                          slot_rels[g.joins[t].b].end());
      TreeNode j;
      j.left = slot_node[g.joins[t].a];
      j.right = slot_node[g.joins[t].b];
      nodes.push_back(j);
      slot_node[s] = (int)nodes.size() - 1;
    }
    // top-down: the largest subtrees that fit are searched exactly
    struct Refine {
      std::vector<TreeNode>& nodes;
      const std::vector<uint64_t>& rmask;
      uint64_t emask;
      int nrel;
      const std::vector<double>& vres;
      int go(int t) {
        if (nodes[t].leaf >= 0) return t;
        std::vector<int> in;
        tree_leaves(nodes, t, in);
        if ((int)in.size() <= kMaxOptimalRelations) {
          uint64_t need = emask;
          for (int i = 0; i < nrel; ++i)
            if (std::find(in.begin(), in.end(), i) == in.end()) need |= rmask[i];
          return exact_tree(in, rmask, need, vres, nodes);
        }
        const int l = go(nodes[t].left), r = go(nodes[t].right);
        nodes[t].left = l;
        nodes[t].right = r;
        return t;
      }
    } refine{nodes, rmask, emask, n, vres};
    root = refine.go(slot_node[g.root]);
  }
  Plan out;
  std::vector<std::vector<int>> slot_vars;
  for (auto& rv : rel_vars) {
    std::vector<int> d;
    for (int v : rv)
      if (std::find(d.begin(), d.end(), v) == d.end()) d.push_back(v);
    slot_vars.push_back(d);
  }
  out.root = emit_plan(nodes, root, n, rel_vars, rmask, emask, vres, slot_vars, out);
  plan = out;
  return true;
}

// policy (order == PA_ORDER_GREEDY): 0 greedy as documented; 1 smallest cost
// r^Lambda first; 2 + seed: at every step a seeded random pick among the three
// best greedy pairs (candidate orders for the learned cost model).
Plan plan_joins_policy(int nvars, const std::vector<double>& vres,
                       const std::vector<std::vector<int>>& rel_vars,
                       const std::vector<int>& exposed, int order, const int32_t* given_pairs,
                       uint64_t policy) {
  uint64_t rng = policy * 0x9E3779B97F4A7C15ull + 0x160900061ull;
  auto next_rand = [&rng]() {
    uint64_t z = (rng += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  };
  Plan plan;
  if (order == PA_ORDER_OPTIMAL) {
    if (plan_optimal(nvars, vres, rel_vars, exposed, plan)) return plan;
    order = PA_ORDER_GREEDY;  // more than 64 variables: the greedy order
  }
  int nrel = (int)rel_vars.size();
  // live slots: slot id -> variable set
  std::vector<std::vector<int>> slot_vars;
  for (auto& rv : rel_vars) {
    std::vector<int> d;
    for (int v : rv)
      if (std::find(d.begin(), d.end(), v) == d.end()) d.push_back(v);
    slot_vars.push_back(d);
  }
  std::vector<int> live;
  for (int i = 0; i < nrel; ++i) live.push_back(i);
  // depth of every slot in the cluster tree (plots 0)
  std::vector<int> depth(nrel, 0);
  (void)nvars;
  auto needed_outside = [&](const std::vector<int>& skip) {
    std::vector<int> need = exposed;
    for (int s : live) {
      if (std::find(skip.begin(), skip.end(), s) != skip.end()) continue;
      need = set_union(need, slot_vars[s]);
    }
    return need;
  };
  auto keep_of = [&](int a, int b) {
    std::vector<int> u = set_union(slot_vars[a], slot_vars[b]);
    std::vector<int> need = needed_outside({a, b});
    std::vector<int> k;
    for (int v : u)
      if (std::find(need.begin(), need.end(), v) != need.end()) k.push_back(v);
    return k;
  };
  for (int t = 0; t < nrel - 1; ++t) {
    int a = -1, b = -1;
    if (order == PA_ORDER_GIVEN) {
      a = given_pairs[2 * t];
      b = given_pairs[2 * t + 1];
    } else if (order == PA_ORDER_LEFT) {
      a = live[0];
      b = live[1];
    } else {
      // smallest result, then smallest cost r^Lambda, then the shallower pair:
      // among equal joins the tree stays balanced, so that independent joins
      // can run side by side (the parallel cost of Sec. 3.5)
      struct Cand {
        double k1, k2;
        int dep, x, y;
      };
      std::vector<Cand> cands;
      for (size_t i = 0; i < live.size(); ++i)
        for (size_t j = i + 1; j < live.size(); ++j) {
          int x = live[i], y = live[j];
          double size = set_size(keep_of(x, y), vres);
          double cost = set_size(set_union(slot_vars[x], slot_vars[y]), vres);
          int dep = std::max(depth[x], depth[y]);
          if (policy == 1) cands.push_back({cost, size, dep, x, y});
          else cands.push_back({size, cost, dep, x, y});
        }
      std::stable_sort(cands.begin(), cands.end(), [](const Cand& p, const Cand& q) {
        if (p.k1 != q.k1) return p.k1 < q.k1;
        if (p.k2 != q.k2) return p.k2 < q.k2;
        return p.dep < q.dep;
      });
      size_t pick = 0;
      if (policy >= 2 && cands.size() > 1) pick = next_rand() % std::min<size_t>(3, cands.size());
      a = cands[pick].x;
      b = cands[pick].y;
    }
    Join jn;
    jn.a = a;
    jn.b = b;
    jn.keep = keep_of(a, b);
    jn.cost = set_size(set_union(slot_vars[a], slot_vars[b]), vres);
    plan.joins.push_back(jn);
    plan.pixel_ops += jn.cost;
    plan.peak_bits = std::max(plan.peak_bits, set_size(jn.keep, vres));
    int id = nrel + t;
    slot_vars.push_back(jn.keep);
    depth.push_back(1 + std::max(depth[a], depth[b]));
    live.erase(std::find(live.begin(), live.end(), a));
    live.erase(std::find(live.begin(), live.end(), b));
    live.insert(live.begin(), id);
    // keep the running product first so PA_ORDER_LEFT folds left to right
  }
  plan.root = live.empty() ? -1 : live[0];
  return plan;
}

bool plan_valid_given(int nrel, int npairs, const int32_t* pairs) {
  if (npairs != nrel - 1 || (nrel > 1 && pairs == nullptr)) return false;
  std::vector<int> used(2 * nrel, 0);
  for (int t = 0; t < npairs; ++t) {
    int a = pairs[2 * t], b = pairs[2 * t + 1];
    int limit = nrel + t;
    if (a < 0 || b < 0 || a >= limit || b >= limit || a == b) return false;
    if (used[a] || used[b]) return false;
    used[a] = used[b] = 1;
  }
  return true;
}

// ------------------------------------------------------------ tree cost
pa_status tree_cost(int32_t nlinks, const double* link_res, int32_t npacks,
                    const int32_t* pack_nports, const int32_t* pack_links, int32_t nouter,
                    const int32_t* outer_links, int32_t njoins, const int32_t* join_nchildren,
                    const int32_t* join_children, double* serial, double* parallel) {
  if (nlinks < 0 || npacks < 1 || njoins < 0 || !serial || !parallel) return PA_ERR_INVALID_ARG;
  int nslots = npacks + njoins;
  // members[s]: packs inside slot s; links[s]: links touched by slot s
  std::vector<std::vector<int>> members(nslots);
  std::vector<std::vector<int>> pack_link_list(npacks);
  int off = 0;
  for (int i = 0; i < npacks; ++i) {
    for (int j = 0; j < pack_nports[i]; ++j) {
      int l = pack_links[off + j];
      if (l < 0 || l >= nlinks) return PA_ERR_INVALID_ARG;
      pack_link_list[i].push_back(l);
    }
    off += pack_nports[i];
    members[i].push_back(i);
  }
  std::vector<double> pcost(nslots, 0.0);
  double total = 0.0;
  int coff = 0;
  // intermediate pack of a slot: its links that touch a pack outside it or the outer pack
  auto inter_pack = [&](int s) {
    std::vector<int> inside(npacks, 0);
    for (int p : members[s]) inside[p] = 1;
    std::vector<int> q;
    for (int p : members[s])
      for (int l : pack_link_list[p]) {
        if (std::find(q.begin(), q.end(), l) != q.end()) continue;
        bool outside = false;
        for (int j = 0; j < nouter && !outside; ++j) outside = (outer_links[j] == l);
        for (int p2 = 0; p2 < npacks && !outside; ++p2) {
          if (inside[p2]) continue;
          outside = std::find(pack_link_list[p2].begin(), pack_link_list[p2].end(), l) !=
                    pack_link_list[p2].end();
        }
        if (outside) q.push_back(l);
      }
    return q;
  };
  for (int t = 0; t < njoins; ++t) {
    int s = npacks + t;
    std::vector<int> links;
    double below = 0.0;
    for (int c = 0; c < join_nchildren[t]; ++c) {
      int ch = join_children[coff + c];
      if (ch < 0 || ch >= s) return PA_ERR_INVALID_ARG;
      for (int p : members[ch]) members[s].push_back(p);
      std::vector<int> q = (ch < npacks) ? pack_link_list[ch] : inter_pack(ch);
      links = set_union(links, q);
      below = std::max(below, pcost[ch]);
    }
    coff += join_nchildren[t];
    // the root is the exterior diagram of the last clustering: its links also
    // include the outer pack's (Sec. 3.5, C-factorization)
    if (t == njoins - 1)
      for (int j = 0; j < nouter; ++j)
        if (std::find(links.begin(), links.end(), outer_links[j]) == links.end())
          links.push_back(outer_links[j]);
    double c = 1.0;
    for (int l : links) c *= link_res[l];
    total += c;
    pcost[s] = c + below;
  }
  *serial = total;
  *parallel = njoins ? pcost[nslots - 1] : 0.0;
  return PA_OK;
}

}  // namespace pa
