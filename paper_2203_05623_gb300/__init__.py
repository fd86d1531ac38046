"""GB300-native batched DFPT response chi0 for plane-wave full-frequency GW.

The compute path is libwgw.so (hand-written sm_103a CUDA kernels behind a C
ABI, declared in include/wgw.h); this package holds its build script and a
thin ctypes binding with the same function names.
"""
from .wgw import (  # noqa: F401
    WGW_ERR_ARG, WGW_ERR_CUDA, WGW_ERR_NOCONV, WGW_ERR_NOMEM, WGW_FP64, WGW_MIXED, WGW_OK,
    WGW_SPHERE_RHO, WGW_SPHERE_WFC, WgwError, lib, wgw_apply_chi0, wgw_apply_chi0_dev,
    wgw_apply_chibar0, wgw_apply_chibar0_dev, wgw_lanczos, wgw_pdep_davidson, wgw_symm_eig_dev, wgw_default_options, wgw_destroy, wgw_get_gvectors,
    wgw_profile_enable, wgw_profile_classes, wgw_profile_read, wgw_set_options, wgw_setup, wgw_system_info,
    wgw_sphere_size, wgw_submit, wgw_submit_pdep, wgw_poll, wgw_wait, wgw_cancel, wgw_dyson, wgw_g0_lanczos, wgw_apply_channels, wgw_pdep_davidson_channels, wgw_selftest_wait_timeout, wgw_apply_h_dev, wgw_autotune_info, wgw_autotune_fft, wgw_autotune_chunk, FFT_KERNEL_NAMES, wgw_sigma_x, wgw_isr, wgw_lanczos_z, wgw_sigma, wgw_qp, wgw_sample_solutions, wgw_read_samples, WGW_REQ_CHI0, WGW_REQ_CHIBAR0, WGW_REQ_PDEP, WGW_ERR_CANCELLED,
)
