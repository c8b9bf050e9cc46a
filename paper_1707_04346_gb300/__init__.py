"""GB300 (sm_103a) determinant-CI sigma = H c and Davidson (arXiv 1707.04346).

The compute lives in ``libfci_gb300.so`` (hand-written CUDA, C ABI declared in
``include/fci.h``); this package only marshals arguments to it.
"""
from .fci import (  # noqa: F401
    FCI_F32, FCI_F64, FCI_PREC_FP64, FCI_PREC_MIXED, FciContext, FciError, default_options, fci_davidson,
    fci_davidson_log, fci_free, fci_get_single_table, fci_get_strings, fci_hdiag, fci_init, fci_profile_enable, fci_profile_read,
    fci_query, fci_rdm1, fci_rdm2, fci_sigma, fci_init_default, fci_free_default, fci_sigma_ptr, load, FciBatch, fci_batch_init, fci_batch_davidson,
    fci_batch_sigma, fci_batch_tuning, fci_batch_stats, fci_batch_free, fci_rdm1_noalloc, fci_tile_schedule,
)
