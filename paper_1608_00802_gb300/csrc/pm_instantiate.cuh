// Explicit instantiations of the precision-templated launchers, shared by the
// fp32 and fp64 translation units.
#pragma once

#define PM_INSTANTIATE(R)                                                                                         \
  template cudaError_t launch_init_particles<R>(const double*, const double*, int64_t, Mesh, double, void*, void*, \
                                                uint32_t*, uint32_t*, cudaStream_t);                              \
  template cudaError_t launch_sort_pass<R>(bool, const uint32_t*, const uint32_t*, int64_t, int, int,             \
                                           const uint32_t*, uint64_t*, uint32_t*, const uint32_t*, int, int,       \
                                           uint32_t*, uint32_t*, const void*, const void*, void*, void*,           \
                                           uint32_t*, cudaStream_t, const uint32_t*, int, size_t, int);           \
  template cudaError_t launch_deposit<R>(const void*, const uint32_t*, int64_t, Mesh, double, R*, cudaStream_t,    \
                                         int, int, size_t);                                                       \
  template cudaError_t launch_resort<R>(int, const uint32_t*, int64_t, const uint32_t*, uint32_t*, uint32_t*, uint32_t*, \
                                        uint32_t*, uint32_t*, uint32_t*, uint32_t*, uint32_t*, uint32_t*, uint32_t*, \
                                        uint32_t*, uint32_t*, Mesh, unsigned long long*, uint32_t*, const void*,     \
                                        const void*, void*, void*, int, cudaStream_t, int, size_t);               \
  template cudaError_t launch_green<R>(void*, Mesh, double, double*, cudaStream_t, const double*, int, size_t);   \
  template cudaError_t launch_spline_weights<R>(void*, Mesh, double, cudaStream_t);                               \
  template cudaError_t launch_spline_symbol<R>(const void*, void*, Mesh, cudaStream_t);                           \
  template cudaError_t launch_green_spline<R>(void*, void*, const void*, Mesh, double, double*, cudaStream_t, int); \
  template cudaError_t launch_smooth_spec<R>(void*, const void*, Mesh, cudaStream_t);                             \
  template cudaError_t launch_stencil<R>(const R*, Mesh, StencilParams, R*, double*, uint32_t*, uint32_t*,       \
                                          uint32_t*, cudaStream_t, const double*, int, size_t);                   \
  template cudaError_t launch_kick<R>(void*, void*, uint32_t*, uint32_t*, int64_t, const R*, const R*, Mesh,      \
                                      KickParams, const KickParams*, const uint32_t*,                              \
                                      double*, double*, uint32_t*, int, cudaStream_t, int, size_t);                \
  template cudaError_t launch_power<R>(const void*, Mesh, int, double*, cudaStream_t);                            \
  template cudaError_t launch_get_particles<R>(const void*, const void*, int64_t, Mesh, double, double*, double*, \
                                               cudaStream_t);                                                     \
  template cudaError_t launch_get_order<R>(const void*, const void*, int64_t, uint32_t*, uint32_t*, cudaStream_t); \
  template cudaError_t launch_to_double<R>(const R*, int64_t, double*, cudaStream_t);                             \
  template cudaError_t launch_from_double<R>(const double*, int64_t, R*, cudaStream_t);
