// Compiled instances of the nodal J.v kernels in double-float arithmetic (FP64 inputs and
// outputs, q scratch as float pairs): quadrilaterals p = 1..4, hexahedra p = 1..6.
#include "ldg_launch.cuh"
#include "ldg_hex_lines.cuh"

namespace ldg {

template <int DIM, int N1, bool CONV> LinFn lin_df_pick() {
  if constexpr (DIM == 3) return &launch_hex<N1, CONV, df, df>;
  else return &launch_lin<DIM, N1, CONV, df, df>;
}

template <int DIM, bool CONV> LinFn lin_df_by_p(int p) {
  switch (p) {
    case 1: return lin_df_pick<DIM, 2, CONV>();
    case 2: return lin_df_pick<DIM, 3, CONV>();
    case 3: return lin_df_pick<DIM, 4, CONV>();
    case 4: return lin_df_pick<DIM, 5, CONV>();
    case 5: if constexpr (DIM == 3) return lin_df_pick<DIM, 6, CONV>(); else return nullptr;
    case 6: if constexpr (DIM == 3) return lin_df_pick<DIM, 7, CONV>(); else return nullptr;
    default: return nullptr;
  }
}

LinFn lin_df_launcher(int dim, int p, bool conv) {
  if (dim == 2) return conv ? lin_df_by_p<2, true>(p) : lin_df_by_p<2, false>(p);
  if (dim == 3) return conv ? lin_df_by_p<3, true>(p) : lin_df_by_p<3, false>(p);
  return nullptr;
}

}  // namespace ldg
