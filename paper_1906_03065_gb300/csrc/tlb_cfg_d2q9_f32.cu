// Instantiation of the driver for one velocity set and storage precision.
#include "tlb_impl.cuh"

ImplBase* make_impl_d2q9_f32() {
  static Impl<D2Q9, TLB_F32> impl;
  return &impl;
}
