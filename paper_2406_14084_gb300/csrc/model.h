// model.h -- host-side access to the cost-model network for the learned planner.
#pragma once

#include <cstddef>
#include <string>

#include "qs.h"

namespace qs {

// Predictions for host rows (rows x nfeat); runs the forward kernel.  Returns a qs_status.
int model_predict(qs_model *m, const float *X, size_t rows, float *y, std::string &err);
int model_nfeat(const qs_model *m);

// Process-wide model for options.planner = QS_PLANNER_LEARNED (NULL = none).
qs_model *default_cost_model();

}  // namespace qs
