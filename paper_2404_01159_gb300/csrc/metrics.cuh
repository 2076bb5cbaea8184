// Scratch and reference point of the hypervolume kernels (k_finalize.cu),
// shared with their host entry point (api.cu).
#pragma once

namespace rvea {

// Scratch (the run's staging area) for a population of N: f1, f2, f3 [N]
// double (the valid members that dominate the reference point, compacted in
// slot order; f3 = 0 and ref3 = 1 when m = 2), vol [N] double, rank3, byF1,
// byF3 [N] int, then the member count.
struct HvScratch {
  double *f1, *f2, *f3, *vol;
  int *rank3, *byF1, *byF3, *count;
};
struct HvRef {
  double r1, r2, r3;
};

}  // namespace rvea
