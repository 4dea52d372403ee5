// hope_stage_dispatch.cu -- (precision, order) dispatch over the instantiation units.
#include "hope_stage.cuh"

namespace hope {
stage_fn stage_entry_d_lo(int k);
stage_fn stage_entry_d_hi(int k);
stage_fn stage_entry_f_lo(int k);
stage_fn stage_entry_f_hi(int k);
vjp_fn vjp_entry_d_lo(int k);
vjp_fn vjp_entry_d_hi(int k);
vjp_fn vjp_entry_f_lo(int k);
vjp_fn vjp_entry_f_hi(int k);
int smem_attr_entry_d_lo(int k);
int smem_attr_entry_d_hi(int k);
int smem_attr_entry_f_lo(int k);
int smem_attr_entry_f_hi(int k);

stage_fn stage_entry(int prec, int k) {
  if (prec == HOPE_FP64) return k <= 7 ? stage_entry_d_lo(k) : stage_entry_d_hi(k);
  return k <= 7 ? stage_entry_f_lo(k) : stage_entry_f_hi(k);
}

vjp_fn vjp_entry(int prec, int k) {
  if (prec == HOPE_FP64) return k <= 7 ? vjp_entry_d_lo(k) : vjp_entry_d_hi(k);
  return k <= 7 ? vjp_entry_f_lo(k) : vjp_entry_f_hi(k);
}

int smem_attr_entry(int prec, int k) {
  int rc;
  if (prec == HOPE_FP64)
    rc = k <= 7 ? smem_attr_entry_d_lo(k) : smem_attr_entry_d_hi(k);
  else
    rc = k <= 7 ? smem_attr_entry_f_lo(k) : smem_attr_entry_f_hi(k);
  return rc < 0 ? HOPE_EINVAL : rc;
}
}  // namespace hope
