// pic_launch.h -- host-callable launch wrappers of the kernels in pic_kernels.cu.
#pragma once
#include "pic_internal.h"

namespace pic {

struct SweepLaunch {
    int fp64, block, ppt, grid, max_N, n_disc, in_buf;
    const Disc* discs;
    Ctl* ctl;
    unsigned long long seed;
    cudaStream_t stream;
};

cudaError_t launch_sweep(const SweepLaunch& L);
int sweep_occupancy(int fp64, int block, int ppt, int max_N, int n_disc);
cudaError_t launch_finalize(int fp64, const Disc* discs, int n_disc, Ctl* ctl, int out_buf, int mode, int max_slices,
                            int max_N, cudaStream_t st);
cudaError_t launch_load(int fp64, const Disc* discs, int n_disc, Ctl* ctl, int buf, unsigned long long seed,
                        int grid_x, cudaStream_t st);
cudaError_t launch_deposit(int fp64, const Disc* discs, int n_disc, const Ctl* ctl, int buf, int max_N, int grid_x,
                           cudaStream_t st);
cudaError_t launch_backkick(int fp64, const Disc* discs, int n_disc, const Ctl* ctl, int buf, int grid_x,
                            cudaStream_t st);
cudaError_t launch_tables(int fp64, int n_pts, int n_proc, double de, double M, const double* se, const double* si,
                          void* Te, void* Ti, unsigned long long* kmax, cudaStream_t st);
cudaError_t launch_sort(int fp64, const Disc* discs, int n_disc, Ctl* ctl, int src, int dst, unsigned* hist,
                        const long long* hoff, unsigned* tot, unsigned* kr, const long long* eoff, int max_N,
                        int grid_x, cudaStream_t st);
cudaError_t launch_repack(int fp64, const Disc* discs, int n_disc, Ctl* ctl, int src, int dst, int grid_x,
                          cudaStream_t st);
// state transfer: cells and the four SoA value arrays (f, vx, vy, vz), in device staging or mapped
// pinned host memory; a null output array of the unpack is skipped
cudaError_t launch_pack_state(int fp64, const Disc* discs, int d, int sp, int buf, long long n, const int32_t* c,
                              const void* const v[4], unsigned* bad, int grid, cudaStream_t st);
cudaError_t launch_unpack_state(int fp64, const Disc* discs, const Ctl* ctl, int d, int sp, int buf, long long cap,
                                int32_t* c, void* const v[4], int grid, cudaStream_t st);
long long sort_tile_chunks(int chunk);
cudaError_t launch_load_profile(int fp64, const Disc* discs, int n_disc, Ctl* ctl, int buf, unsigned long long seed,
                                const void* warm, int grid_x, cudaStream_t st);
size_t warm_desc_bytes(int fp64);
void warm_desc_fill(int fp64, void* out, const void* cdf_e, const void* cdf_i, const void* eps, int P, double scale,
                    double K23);
cudaError_t launch_diag(int fp64, const Disc* discs, int n_disc, const Ctl* ctl, int buf, const DiagArgs& A,
                        int max_N, int grid_x, cudaStream_t st);
size_t diag_smem(int max_N, unsigned mask, int bins);  // bins: 0 unless the launch samples the EEDF
cudaError_t launch_set_dense(const Disc* discs, int n_disc, Ctl* ctl, int buf, cudaStream_t st);
cudaError_t launch_finish_upload(const Disc* discs, Ctl* ctl, int d, int sp, long long n, const unsigned* bad,
                                 int buf, cudaStream_t st);
cudaError_t launch_debug_wait(int arrive, int tries, int* out, cudaStream_t st);
cudaError_t launch_debug_philox(long long n, const uint32_t* ctr, uint32_t k0, uint32_t k1, uint32_t* out,
                                cudaStream_t st);
cudaError_t launch_debug_math(long long n, const float* x, const float* y, float* lg, float* sn, float* cs,
                              cudaStream_t st);

}  // namespace pic
