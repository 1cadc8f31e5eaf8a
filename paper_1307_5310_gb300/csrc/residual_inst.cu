// One translation unit per spatial degree P (compiled with -DSTM_P=<P>):
// instantiates the residual kernels of residual.cuh for q = 1..6 and both
// precisions, so the build can compile the degrees in parallel.
#include "residual.cuh"

#ifndef STM_P
#error "compile with -DSTM_P=<spatial degree>"
#endif

namespace stm {

template <typename T>
int launch_residual_p(int Q, const ApplyArgs<T>& a, cudaStream_t s, int grid, const LaunchEvents& ev, int phase,
                      int block);

#define STM_CAT2(x, y) x##y
#define STM_CAT(x, y) STM_CAT2(x, y)

template <typename T>
int STM_CAT(launch_residual_p, STM_P)(int Q, const ApplyArgs<T>& a, cudaStream_t s, int grid, const LaunchEvents& ev,
                                      int phase, int block) {
  switch (Q) {
    case 1: return launch_residual_pq<T, STM_P, 1>(a, s, grid, ev, phase, block);
    case 2: return launch_residual_pq<T, STM_P, 2>(a, s, grid, ev, phase, block);
    case 3: return launch_residual_pq<T, STM_P, 3>(a, s, grid, ev, phase, block);
    case 4: return launch_residual_pq<T, STM_P, 4>(a, s, grid, ev, phase, block);
    case 5: return launch_residual_pq<T, STM_P, 5>(a, s, grid, ev, phase, block);
    case 6: return launch_residual_pq<T, STM_P, 6>(a, s, grid, ev, phase, block);
    default: return -1;
  }
}

template int STM_CAT(launch_residual_p, STM_P)<double>(int, const ApplyArgs<double>&, cudaStream_t, int,
                                                          const LaunchEvents&, int, int);
template int STM_CAT(launch_residual_p, STM_P)<float>(int, const ApplyArgs<float>&, cudaStream_t, int,
                                                         const LaunchEvents&, int, int);

}  // namespace stm
