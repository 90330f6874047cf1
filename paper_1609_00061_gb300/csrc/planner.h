// Join planning (Sec. 3.5 clustering) for the pixel array engine; host only.
#pragma once

#include <vector>

#include "pa_internal.h"

namespace pa {

// One pairwise cluster: slots a and b are joined; the result keeps `keep`.
struct Join {
  int a, b;
  std::vector<int> keep;
  double cost;  // r^(variables of a and b): the naive cost of this cluster
};

struct Plan {
  std::vector<Join> joins;
  int root = -1;
  double pixel_ops = 0.0;
  double peak_bits = 0.0;
};

// Joins for relations with the given (distinct-ified) variables.  Slots
// 0..nrel-1 are the relations; join t creates slot nrel + t.
Plan plan_joins(int nvars, const std::vector<double>& vres,
                const std::vector<std::vector<int>>& rel_vars, const std::vector<int>& exposed,
                int order, const int32_t* given_pairs);
Plan plan_joins_policy(int nvars, const std::vector<double>& vres,
                       const std::vector<std::vector<int>>& rel_vars,
                       const std::vector<int>& exposed, int order, const int32_t* given_pairs,
                       uint64_t policy);
bool plan_valid_given(int nrel, int npairs, const int32_t* pairs);

// The pairwise cluster tree of least naive cost (PA_ORDER_OPTIMAL): exact up
// to kMaxOptimalRelations relations; beyond, the greedy tree with every
// subtree of at most that many relations searched exactly.  False when the
// network has more than 64 variables.
constexpr int kMaxOptimalRelations = 16;
bool plan_optimal(int nvars, const std::vector<double>& vres,
                  const std::vector<std::vector<int>>& rel_vars, const std::vector<int>& exposed,
                  Plan& plan);

pa_status tree_cost(int32_t nlinks, const double* link_res, int32_t npacks,
                    const int32_t* pack_nports, const int32_t* pack_links, int32_t nouter,
                    const int32_t* outer_links, int32_t njoins, const int32_t* join_nchildren,
                    const int32_t* join_children, double* serial, double* parallel);

}  // namespace pa
