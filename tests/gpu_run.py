"""Helpers that drive the CUDA library through its C ABI for the GPU tests."""
import numpy as np

import paper_1307_5700_gb300 as tp
from oracle import oracle as O


def rfi_params(rfi):
    """tp_rfi_params from the oracle's RfiParams (same field meanings)."""
    p = tp.tp_rfi_defaults()
    p.enable_channel = int(rfi.enable_channel)
    p.enable_spectrum = int(rfi.enable_spectrum)
    p.chunk_width = int(rfi.chunk_width)
    p.dilate_channels = int(rfi.dilate_channels)
    p.tau_channel = float(rfi.tau_channel)
    p.tau_spectrum = float(rfi.tau_spectrum)
    return p


class GpuBeam:
    """One engine + plan + beam; push blocks and collect every product."""

    def __init__(self, nchan, f_lo, bw, t_samp, dms, dtype, rfi=None, nsigma=5.0, block=None,
                 cap=1 << 16, external=False, engine=None):
        self.own = engine is None
        self.e = engine if engine is not None else tp.tp_engine_create(0)
        rp = rfi_params(rfi or O.RfiParams())
        if external:
            rp.stats_mode = tp.TP_STATS_EXTERNAL
        self.dtype = dtype
        self.nchan = nchan
        self.ndm = len(dms)
        self.plan = tp.tp_create_plan(self.e, nchan, f_lo, bw, t_samp, dms, dtype, rp, nsigma)
        self.info = tp.tp_plan_info(self.plan)
        self.cap = cap
        self.block = block
        self.beam = None

    def open(self, block):
        self.block = block
        self.beam = tp.tp_beam_open(self.e, self.plan, block, self.cap)
        return self

    def run(self, x, fetch=True):
        """Push one block (host numpy array or device tensor) and run A1-A7."""
        if self.beam is None:
            self.open(x.shape[1])
        tp.tp_push_block(self.e, self.beam, x)
        tp.tp_dedisperse(self.e, self.beam)
        tp.tp_detect(self.e, self.beam)
        cands, n, rc = tp.tp_get_candidates(self.e, self.beam, self.cap)
        out = dict(candidates=cands, n_candidates=n, rc=rc, info=tp.tp_beam_info(self.e, self.beam))
        if fetch:
            out["D"] = tp.tp_get_series(self.e, self.beam, ndm=self.ndm, is_int=self.dtype == "u8")
            out["mu"], out["sigma"] = tp.tp_get_bandpass(self.e, self.beam, self.nchan)
            out["chunk_flag"], out["chunk_raw"], out["spec_flag"] = tp.tp_get_masks(self.e, self.beam, self.nchan)
            out["row_mu"], out["row_sigma"] = tp.tp_get_series_stats(self.e, self.beam, self.ndm)
        return out

    def delays(self):
        return tp.tp_get_delay_table(self.plan)

    def close(self):
        if self.beam is not None:
            tp.tp_beam_close(self.e, self.beam)
            self.beam = None
        tp.tp_plan_destroy(self.plan)
        if self.own:
            tp.tp_engine_destroy(self.e)
