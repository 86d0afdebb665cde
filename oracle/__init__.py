"""FP64 CPU oracle of the dual-polarisation coherent receiver chain.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this
package: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may use it.  It shares no code, tables or constants
with the CUDA receiver in ``paper_2108_07001_gb300/``; both are fed the
same seeded samples from ``rxsim``.

Every function states the step it implements.  The paper (arXiv
2108.07001) grounds the overall structure: frequency-domain overlap-save
processing with the overlap carried between buffers and chromatic-dispersion
compensation in the frequency domain (Sec. II), a decision-directed LMS
time-domain equaliser followed by decisions and demapping (Sec. II), and
BER-derived Q-factor (Sec. III).  It is silent on polarisation
demultiplexing, CMA, frequency-offset and timing recovery and blind phase
search; for those the oracle writes out the textbook definition of each
estimator and the schedule fixed for this receiver; where the paper is
silent, the reading taken is stated in the docstring of the function that
takes it.

Parity status per function is given in ``rx_oracle.PIN_STATUS``.
"""
from .rx_oracle import (RxConfig, Geometry, geometry, cd_frequency_response,
                        ols_cd, full_length_cd, godard_sum, foe_block_periodogram,
                        foe_from_periodogram, mimo_fir, sub_block_update,
                        acquire, bps, unwrap_increments, decide, demap, const_map,
                        prbs31_bits, ber_sync, ber_count, Receiver, PIN_STATUS)

__all__ = ["RxConfig", "Geometry", "geometry", "cd_frequency_response", "ols_cd",
           "full_length_cd", "godard_sum", "foe_block_periodogram",
           "foe_from_periodogram", "mimo_fir", "sub_block_update", "acquire", "bps",
           "unwrap_increments", "decide", "demap", "const_map", "prbs31_bits",
           "ber_sync", "ber_count", "Receiver", "PIN_STATUS"]
