// Host-side launchers of the device kernels (one translation unit per
// precision for the step kernel so that the large unrolled bodies compile in
// parallel).
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "lbm_device.cuh"

namespace lbgm {

struct InitInst;

cudaError_t launch_step_f64(int K, const double* fin, double* fout, const GeoDev<double>& geo,
                            const InstParams<double>* inst, const Dims& d, int* flag, int threads,
                            cudaStream_t s);
cudaError_t launch_step_f32(int K, const float* fin, float* fout, const GeoDev<float>& geo,
                            const InstParams<float>* inst, const Dims& d, int* flag, int threads,
                            cudaStream_t s);
cudaError_t launch_step_h16(int K, const __half* fin, __half* fout, const GeoDev<float>& geo,
                            const InstParams<float>* inst, const Dims& d, int* flag, int threads,
                            cudaStream_t s);
cudaError_t launch_step_b16(int K, const __nv_bfloat16* fin, __nv_bfloat16* fout, const GeoDev<float>& geo,
                            const InstParams<float>* inst, const Dims& d, int* flag, int threads,
                            cudaStream_t s);

// Plain step whose instances may use the half-force velocity variant
// (InstParams::pad = 1); see step_shift.cu.
cudaError_t launch_step_shift_f64(int K, const double* fin, double* fout, const GeoDev<double>& geo,
                                  const InstParams<double>* inst, const Dims& d, int* flag, int threads,
                                  cudaStream_t s);
cudaError_t launch_step_shift_f32(int K, const float* fin, float* fout, const GeoDev<float>& geo,
                                  const InstParams<float>* inst, const Dims& d, int* flag, int threads,
                                  cudaStream_t s);

// Region-split step (periodic x3): wall layers on stream se, interior on s.
cudaError_t launch_step_split_f64(int K, const double* fin, double* fout, const GeoDev<double>& geo,
                                  const InstParams<double>* inst, const Dims& d, int* flag, int threads,
                                  cudaStream_t s, cudaStream_t se);
cudaError_t launch_step_split_f32(int K, const float* fin, float* fout, const GeoDev<float>& geo,
                                  const InstParams<float>* inst, const Dims& d, int* flag, int threads,
                                  cudaStream_t s, cudaStream_t se);
cudaError_t launch_step_split_h16(int K, const __half* fin, __half* fout, const GeoDev<float>& geo,
                                  const InstParams<float>* inst, const Dims& d, int* flag, int threads,
                                  cudaStream_t s, cudaStream_t se);
cudaError_t launch_step_split_b16(int K, const __nv_bfloat16* fin, __nv_bfloat16* fout, const GeoDev<float>& geo,
                                  const InstParams<float>* inst, const Dims& d, int* flag, int threads,
                                  cudaStream_t s, cudaStream_t se);

// Work-list step over instances of different geometry (ListInst<S, R> array);
// walls bits 0-1: 0 interior tiles, 1 r-layer wall nodes, 2 x3-layer wall
// nodes, 3 other wall nodes (1..3 over `cells`); bit 2: interior tiles
// longer than one block; grid 0 launches one block per work item.
cudaError_t launch_step_list_f64(int K, int walls, const void* insts, const int4* work, int nwork,
                                 const int* cells, int threads, int grid, int parity, cudaStream_t s);
cudaError_t step_list_occupancy_f64(int K, int threads, int* blocks_per_sm);
int step_list_max_threads_f64();
cudaError_t launch_step_list_f32(int K, int walls, const void* insts, const int4* work, int nwork,
                                 const int* cells, int threads, int grid, int parity, cudaStream_t s);
cudaError_t step_list_occupancy_f32(int K, int threads, int* blocks_per_sm);
int step_list_max_threads_f32();
cudaError_t launch_step_list_h16(int K, int walls, const void* insts, const int4* work, int nwork,
                                 const int* cells, int threads, int grid, int parity, cudaStream_t s);
cudaError_t step_list_occupancy_h16(int K, int threads, int* blocks_per_sm);
int step_list_max_threads_h16();
cudaError_t launch_step_list_b16(int K, int walls, const void* insts, const int4* work, int nwork,
                                 const int* cells, int threads, int grid, int parity, cudaStream_t s);
cudaError_t step_list_occupancy_b16(int K, int threads, int* blocks_per_sm);
int step_list_max_threads_b16();

// TMA-pipelined FP32 step (n3 in {128, 256}); map is a CUtensorMap over the
// input state (make_state_tensor_map).
bool tma_step_supported(const Dims& d);
size_t tensor_map_bytes();
cudaError_t make_state_tensor_map(void* map_out, const float* base, const Dims& d);
cudaError_t launch_step_tma_f32(int K, const void* map, const float* fin, float* fout,
                                const GeoDev<float>& geo, const InstParams<float>* inst, const Dims& d,
                                int* flag, cudaStream_t s);

// prec: 0 = FP64, 1 = FP32, 2 = FP16 deviations, 3 = BF16 deviations (state
// pointers of the storage type; geo a GeoDev<double> for FP64, else GeoDev<float>)
cudaError_t launch_macros(int prec, int K, const void* fin, double* rho, double* u, const Dims& d,
                          cudaStream_t s);
cudaError_t launch_init(int prec, int K, void* f, const void* geo, const double* sqrtg,
                        const double* base_uth, const InitInst* ini, const double* rho_in,
                        const double* u_in, const Dims& d, cudaStream_t s);
cudaError_t launch_convert(int prec, int to_double, void* state, double* dbl, size_t n, const Dims& d,
                           cudaStream_t s);
// Per instance max |u - u_prev| and max |u| into out[2 b], out[2 b + 1];
// u_prev = u afterwards (partial: batch * nblk * 2 doubles).
cudaError_t launch_residual(const double* u, double* u_prev, const Dims& d, double* partial, int nblk,
                            double* out, cudaStream_t s);
// Reference table from the row means of FP64 populations (k_ref_from_state).
cudaError_t launch_ref_from_state(const double* dbl, float* ref, const Dims& d, cudaStream_t s);
// Reference populations of 2-byte storage (k_ref_table): mode 0 weights,
// 1 the initial rows' equilibria (from the row means of rho_in / u_in if
// given, else base_uth, which may be NULL: rest).
cudaError_t launch_ref_table(int K, float* ref, const GeoDev<float>& geo, const double* sqrtg,
                             const double* base_uth, const double* rho_in, const double* u_in, const Dims& d,
                             int mode, cudaStream_t s);

// Stream table of 2-byte storage (k_stream_table) from the reference table
// and the instances' omega; prec 2 (FP16) or 3 (BF16), fin any state block.
cudaError_t launch_stream_table(int prec, int K, float4* st, const float* ref, const InstParams<float>* inst,
                                const void* fin, const Dims& d, cudaStream_t s);

// Observables: NQ sums per instance written to out[batch * DIAG_NQ].
constexpr int DIAG_NQ = 9;
cudaError_t launch_diag(const double* rho, const double* u, double* rowmean, const double* geo64,
                        const Dims& d, double* partial, int nblk, double* out, cudaStream_t s);

// Message for lb_last_error(NULL) from entry points without a context.
void set_last_error_noctx(const std::string& msg);

}  // namespace lbgm
