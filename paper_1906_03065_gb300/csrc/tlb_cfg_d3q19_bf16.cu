// Instantiation of the driver for one velocity set and storage precision.
#include "tlb_impl.cuh"

ImplBase* make_impl_d3q19_bf16() {
  static Impl<D3Q19, TLB_BF16> impl;
  return &impl;
}
