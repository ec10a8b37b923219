// Host launchers of the U-Net layer kernels (unet.cu), called by the C ABI in unet.cu.
#pragma once

#include <cuda_runtime.h>

namespace eptv {

extern thread_local long long g_launch_count;   // kernels launched on this thread (cgls.cu)

bool unet_conv_supported(int cin, int cout);
// tensor-memory (tcgen05) path of the 3x3 conv (unet_tc.cu): cudaErrorNotSupported for
// image widths it does not tile; and its error flag (1: a bounded wait ran out)
cudaError_t unet_conv3x3_tc(const void *x, int n, int H, int W, int cin, int xs, int xo, const void *wt,
                            const float *b, int cout, void *y, int ys, int yo, int relu, cudaStream_t st,
                            bool all_shapes);
cudaError_t unet_tc_status(int *flag);
cudaError_t unet_conv3x3(const void *x, int n, int H, int W, int cin, int xs, int xo, const void *wt,
                         const float *b, int cout, void *y, int ys, int yo, int relu, cudaStream_t st);
cudaError_t unet_conv3x3_wgrad(const void *x, int n, int H, int W, int cin, int xs, int xo,
                               const void *dy, int dys, int dyo, int cout, float *dw, float *db,
                               cudaStream_t st);
cudaError_t unet_weights_to_bf16(const float *w, int cout, int cin, void *wf, void *wb, cudaStream_t st);
cudaError_t unet_maxpool2(const void *x, int n, int H, int W, int xs, int xo, int C, void *y, int ys,
                          int yo, cudaStream_t st);
cudaError_t unet_maxpool2_bwd(const void *x, int n, int H, int W, int xs, int xo, int C, const void *dy,
                              int dys, int dyo, void *dx, int dxs, int dxo, int acc, cudaStream_t st);
cudaError_t unet_upsample2(const void *x, int n, int H, int W, int xs, int xo, int C, void *y, int ys,
                           int yo, cudaStream_t st);
cudaError_t unet_upsample2_bwd(const void *dy, int n, int H, int W, int dys, int dyo, int C, void *dx,
                               int dxs, int dxo, cudaStream_t st);
cudaError_t unet_relu_bwd(const void *a, int as, int ao, const void *dy, int dys, int dyo, void *dz,
                          int dzs, int dzo, long long npix, int C, cudaStream_t st);
cudaError_t unet_head(const void *x, int xs, int xo, long long npix, const float *hw, const float *hb,
                      float *f0, float *w, const float *base, float f_scale, const float *ft,
                      const float *wt, void *dx, int dxs, int dxo, float *dhw, float *dhb, double *loss,
                      cudaStream_t st);
cudaError_t unet_pack_input(const float *a, float sa, const float *b, float sb, long long npix, void *x,
                            cudaStream_t st);
cudaError_t unet_adam(float *p, const float *g, float *m, float *v, long long n, float lr, float b1,
                      float b2, float eps, int step, cudaStream_t st);


}  // namespace eptv
