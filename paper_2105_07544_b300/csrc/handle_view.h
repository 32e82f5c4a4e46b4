// Read-only view of a solver handle's device matrix for library code outside solver.cu (the
// controller's feature kernels).  Not part of the public C ABI.
#pragma once

#include <cstdint>

#include "../../include/gmresb3.h"

namespace gmresb3 {

struct HandleView {
  int64_t n, nnz;
  const int32_t* rowptr;   // device, n + 1 entries
  const int32_t* col;      // device, nnz entries
  const double* val;       // device, nnz FP64 values
  int dev;                 // device the handle was created on
  int sms;                 // its streaming multiprocessors
  void* user_stream;       // the caller's stream set with gmres_set_stream (NULL = legacy)
};

HandleView handle_view(gmres_handle_t h);

}  // namespace gmresb3
