// Compiled instances of the nodal J.v kernels in double-float arithmetic (FP64 inputs and
// outputs, q scratch as float pairs): quadrilaterals p = 1..4, hexahedra p = 1..6.
#include "ldg_launch.cuh"
#include "ldg_hex_lines.cuh"

namespace ldg {

template <int DIM, int N1, bool CONV> LinFn lin_df_pick(bool cart) {
  if constexpr (DIM == 3) return cart ? &launch_hex<N1, CONV, df, df, true> : &launch_hex<N1, CONV, df, df, false>;
  else return cart ? &launch_lin<DIM, N1, CONV, df, df, true> : &launch_lin<DIM, N1, CONV, df, df, false>;
}

template <int DIM, bool CONV> LinFn lin_df_by_p(int p, bool cart) {
  switch (p) {
    case 1: return lin_df_pick<DIM, 2, CONV>(cart);
    case 2: return lin_df_pick<DIM, 3, CONV>(cart);
    case 3: return lin_df_pick<DIM, 4, CONV>(cart);
    case 4: return lin_df_pick<DIM, 5, CONV>(cart);
    case 5: if constexpr (DIM == 3) return lin_df_pick<DIM, 6, CONV>(cart); else return nullptr;
    case 6: if constexpr (DIM == 3) return lin_df_pick<DIM, 7, CONV>(cart); else return nullptr;
    default: return nullptr;
  }
}

LinFn lin_df_launcher(int dim, int p, bool conv, bool cart) {
  if (dim == 2) return conv ? lin_df_by_p<2, true>(p, cart) : lin_df_by_p<2, false>(p, cart);
  if (dim == 3) return conv ? lin_df_by_p<3, true>(p, cart) : lin_df_by_p<3, false>(p, cart);
  return nullptr;
}

}  // namespace ldg
