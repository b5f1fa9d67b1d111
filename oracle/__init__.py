"""CPU FP64 oracle for the partitioned tile-program hot path.

TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check of the package entry
and the CPU-baseline leg of the benchmark may import this package. The product
path (the CUDA library and its Python binding) never imports it, and this
package imports nothing from the product path: the two share no code. The only
module both sides use is `synth`, which draws the seeded inputs and holds none
of the method's arithmetic.

Every function states its result by its plain definition (the paper's, or the
format's), in float64 unless a precision is fixed by the operation itself
(a quantised code is decided in the precision the kernel uses, fp32).

Modules
  lowp       bf16 / fp8-E4M3 rounding from the format definitions
  maps       element-wise maps (axpy, gelu_tanh * w)
  gemm       FP64 GEMM, bf16 output rounding, per-tensor-scaled FP8 GEMM
  partition  tile grids, tile->program maps, write-count checker
  grouped    grouped GEMM problems and tile-queue coverage
  decode     batch-1 decode-shaped chain (RMSNorm, GEMVs, SiLU*mul, residual)
  mlp        3-layer MLP forward / backward / Adam for the tile proposer
"""
