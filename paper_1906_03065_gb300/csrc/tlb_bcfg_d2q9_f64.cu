// Instantiation of the batched driver for one velocity set and storage precision.
#include "tlb_batch.cuh"

static_assert(sizeof(BArgs<TLB_F64>) <= Batch::ARGS_BYTES, "instance argument record too large");

BatchBase* make_batch_impl_d2q9_f64() {
  static BatchImpl<D2Q9, TLB_F64> impl;
  return &impl;
}
