"""Seeded synthetic inputs for the SALT photometry path (shared by the tests,
the oracle checks and the bench; no photometry arithmetic lives here)."""
from .synth import (Band, Batch, Model, Request, Workload, add_noise, config1, config2,
                    config3, config4, config5, gaussian_band, make, make_batch, make_model,
                    subset, template_flux, tophat_band, truth_batch, fit_start, CONFIG_NAMES, PERTURB,
                    FIT_PERTURB, config_nir, make_model_nodes, NIR_PHASE_NODES, NIR_WAVE_NODES)
