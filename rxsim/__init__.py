"""Seeded synthetic optical-link generator for the coherent receiver.

This package produces the *inputs* of the receiver: dual-polarisation
received samples of a Gray-coded QPSK/16QAM signal after a transmitter,
a fibre and a receiver front end, together with the transmitted bits.
It models the forward channel only (transmitter pulse shaping, a random
unitary polarisation rotation, chromatic dispersion, a sampling-clock
delay, a laser frequency offset with Wiener phase noise and AWGN); it
contains no part of the receiver's signal processing.  ``simulate_kk``
generates the single-polarisation minimum-phase signal (carrier tone plus
QAM) that the paper detects with one photodiode for its Kramers-Kronig
front end, as 12-bit ADC codes.  Both the FP64
oracle (``oracle/``) and the CUDA receiver are fed from here, and neither
imports anything else from the other.
"""
from .channel import (LinkConfig, simulate, prbs31, pol_seed_state, gray_map,
                      C_LIGHT, beta2_from_dispersion)
from .kk import KKLinkConfig, simulate_kk

__all__ = ["LinkConfig", "simulate", "prbs31", "pol_seed_state", "gray_map",
           "C_LIGHT", "beta2_from_dispersion", "KKLinkConfig", "simulate_kk"]
