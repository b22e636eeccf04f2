// Schwarz alternating procedure (csrc/sap.cu): the preconditioner's parameters and entry point.
#pragma once

#include "qxd_internal.cuh"

namespace qxd {

struct SapSpec {
  int block[4];  // block extents (each divides the lattice; an even number of blocks per direction)
  int ncy;       // cycles from zero
  int nmr;       // minimal-residual steps per block solve
};

// z = M_SAP r on full FP32 fields in the internal layout (work slots 41, 42)
qxd_status sap32(qxd_lattice* lat, const int b[4], int ncy, int nmr, const float4* rin, float4* z);

}  // namespace qxd
