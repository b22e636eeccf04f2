// Schwarz alternating procedure (csrc/sap.cu): the preconditioner's parameters and entry point.
#pragma once

#include "qxd_internal.cuh"

namespace qxd {

struct SapSpec {
  int block[4];  // block extents (each divides the lattice; an even number of blocks per direction)
  int ncy;       // cycles from zero
  int nmr;       // minimal-residual steps per block solve
  int dfl = 0;   // 1: two-level preconditioner (deflation coarse solve, then SAP), csrc/dfl.cu
  int mg = 0;    // 1: three-level multigrid preconditioner, csrc/mg.cu
};

// z = M_SAP r on full FP32 fields in the internal layout (work slots 41, 42)
qxd_status sap32(qxd_lattice* lat, const int b[4], int ncy, int nmr, const float4* rin, float4* z);
qxd_status sap_check(qxd_lattice* lat, const int b[4]);

// Two-level preconditioner of DFL_SAP_GCR (csrc/dfl.cu): z = P A^-1 P^+ r (coarse solve on the
// deflation subspace set up by qxd_dfl_setup), then z += M_SAP (r - D z).  Full FP32 fields.
qxd_status dfl_precond32(qxd_lattice* lat, const SapSpec& sap, const float4* r, float4* z);
bool dfl_ready(const qxd_lattice* lat);

// The multigrid preconditioner of MG_GCR (csrc/mg.cu): z = M_SAP^pre r; z += P1 K1(P1^+ (r - D z));
// z += M_SAP (r - D z), with K1 the level-1 K-cycle over the aggregation of qxd_mg_setup.
qxd_status mg_precond32(qxd_lattice* lat, const SapSpec& sap, const float4* r, float4* z);
bool mg_ready(const qxd_lattice* lat);

}  // namespace qxd
