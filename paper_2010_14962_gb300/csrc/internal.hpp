// Internal access to plan handles for translation units other than the
// C-ABI layer (not part of the public interface).
#pragma once
#include <mutex>
#include <string>

#include "../../include/qtn.h"
#include "program.hpp"

namespace qtn {
namespace internal {

struct PlanView {
  const Program* program;  // the program of the plan's executor
  bool lane;               // executor: lane (true) or block (false)
  bool wide;               // the per-slice program is a wide (global-memory) one
  int n;                   // qubits
  int k;                   // cuts
  const double* gamma;     // host, p entries
  const double* beta;
  int p;
  std::mutex* mu;          // serialises contraction calls on the plan
};

// Fills `view` for `plan`; returns false if plan is NULL.
bool plan_view(const qtn_plan_t* plan, PlanView* view);

// The host network behind a handle.
const Network* network_of(const qtn_network_t* net);

// Sets the calling thread's qtn_last_error() text and returns `s`.
qtn_status set_error(qtn_status s, const std::string& msg);

}  // namespace internal
}  // namespace qtn
