"""Seeded synthetic inputs shared by the CUDA path's tests and benches and by
the CPU oracle's tests: parity-check matrices, codewords and AWGN channel
values.  Nothing here performs a step of the decoding method."""
from .codes import (ParityCheck, eg2_cyclic, eg2_offsets, quasi_cyclic,
                    random_qc, random_regular, primitive_polynomial)
from .gf2 import Encoder, gf2_rank
from .channel import awgn_sigma, bpsk_awgn, random_codewords
from .workloads import WORKLOADS, make_code
