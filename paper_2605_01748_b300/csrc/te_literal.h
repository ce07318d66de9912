// Internal declaration of the printed multi-block iteration (te_literal.cu),
// behind te_literal_run of include/te.h.
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "te.h"

namespace te {

// Runs iters iterations of the printed update equations from Algorithm 1's
// start on the checked instance (host arrays) and writes the rates in
// caller units to x_out (host, [n_paths]).  Device memory is allocated for
// the call and released before it returns; st is synchronised.
te_status literal_run(const te_paths* P, int n_edges, const double* demands, const double* capacities, double alpha,
                      double beta, long long iters, double* x_out, cudaStream_t st, std::string& err);

}  // namespace te
