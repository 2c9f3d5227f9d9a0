// learned.h -- candidate-plan selection by the cost model (learned.cpp).
#pragma once

#include <string>
#include <vector>

#include "planner.h"

namespace qs {

struct LearnedMeta {
    int candidates = 0;        // distinct plans scored (the greedy plan included)
    int chosen = -1;           // grid index of the chosen candidate; -1 = greedy kept
    double predicted_ms = 0;   // prediction for the returned plan
    double greedy_ms = 0;      // prediction for the greedy plan
};

// Build the greedy plan for `opt` into `greedy`; with a model, also score the candidate grid
// and, when one is predicted >= 5% faster, move it into `best` (meta.chosen >= 0).
int learned_choose(const std::vector<CGate> &gates, int n, qs_dtype dt, const qs_options &opt, qs_model *model,
                   Plan &greedy, Plan &best, LearnedMeta &meta, std::string &err);

}  // namespace qs
