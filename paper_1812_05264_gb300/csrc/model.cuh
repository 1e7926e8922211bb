// Device-side copy of a tbk_model (plain values plus device pointers).
#pragma once
#include "common.cuh"

namespace tbk {

struct DevModel {
  int kind, n_orb;
  double V[10], r0, decay, onsite[3];
  double box[3];
  int n_disp;
  double tol;
  const double* disp;        // device, n_disp x 3
  const double* blocks;      // device, n_disp x n_orb^2
  const double* onsite_site; // device, n_atoms x n_orb, or NULL
};

// Validate `model` and copy its tables to device scratch slot `slot`.
DevModel upload_model(tbk_ctx* ctx, const tbk_model* model, const double* box, Slot slot);

}  // namespace tbk
