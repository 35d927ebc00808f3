"""GB300-native (sm_103a) CP-ALS-QR hot path: Multi-TTM, structured QR of the
Khatri-Rao product, Q0 application, triangular/SVD solves, MTTKRP baseline and
fit, as hand-written CUDA behind a C-ABI library (libcpals.so)."""
