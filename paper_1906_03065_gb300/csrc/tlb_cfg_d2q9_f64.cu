// Instantiation of the driver for one velocity set and storage precision.
#include "tlb_impl.cuh"

ImplBase* make_impl_d2q9_f64() {
  static Impl<D2Q9, TLB_F64> impl;
  return &impl;
}
