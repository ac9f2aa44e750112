// mlq_host.h -- host helpers shared between translation units of the library
// (not part of the C ABI).
#pragma once

#include <cstdint>

namespace mlq {

// The simplex of a general mesh (xyz n x dim, conn ne x (dim + 1)) holding
// each point of pts (np x dim) and the point's barycentric coordinates there
// (mlq_kl.cpp): elem np, lam np x (dim + 1).  The first simplex in element
// order that contains the point; a point in no simplex takes the first one
// whose smallest coordinate is within 1e-12 of the largest over all
// simplices.  MLQ_OK or MLQ_EINVAL.
int locate_points(int dim, int64_t n, const double *xyz, int64_t ne, const int32_t *conn, int64_t np,
                  const double *pts, int64_t *elem, double *lam);

}  // namespace mlq
