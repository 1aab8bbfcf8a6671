// Compiled instances of the nodal J.v kernels in double-float arithmetic (FP64 inputs and
// outputs, q scratch as float pairs): quadrilaterals p = 1..4, hexahedra p = 1..6.
#include "ldg_launch.cuh"
#include "ldg_linear.cuh"

namespace ldg {

template <int DIM, bool CONV> LinFn lin_df_by_p(int p) {
  switch (p) {
    case 1: return &launch_lin<DIM, 2, CONV, df, df>;
    case 2: return &launch_lin<DIM, 3, CONV, df, df>;
    case 3: return &launch_lin<DIM, 4, CONV, df, df>;
    case 4: return &launch_lin<DIM, 5, CONV, df, df>;
    case 5: if constexpr (DIM == 3) return &launch_lin<DIM, 6, CONV, df, df>; else return nullptr;
    case 6: if constexpr (DIM == 3) return &launch_lin<DIM, 7, CONV, df, df>; else return nullptr;
    default: return nullptr;
  }
}

LinFn lin_df_launcher(int dim, int p, bool conv) {
  if (dim == 2) return conv ? lin_df_by_p<2, true>(p) : lin_df_by_p<2, false>(p);
  if (dim == 3) return conv ? lin_df_by_p<3, true>(p) : lin_df_by_p<3, false>(p);
  return nullptr;
}

}  // namespace ldg
