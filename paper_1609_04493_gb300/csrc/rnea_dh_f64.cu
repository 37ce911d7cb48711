// rnea_dh_f64.cu -- double instantiations of the common-normal-frame RNEA kernels.
#include "rnea_dh_launch.cuh"

int rd_rnea_dh_f64(const rd_model *m, int B, const void *q, const void *qd, const void *qdd,
                   void *tau, const double *base18, int stored, int block, int fast,
                   int kfull, int tmem, int reg_links, int stages, cudaStream_t s)
{
    return rdyn::dh_launch<double>(m, B, q, qd, qdd, tau, base18, stored != 0, block, false, kfull, tmem != 0, reg_links, stages, s);
}
