"""Domain decomposition of the field update along z with guard cells, on one GPU.

The finite-order stencil of the paper reaches only a finite number of cells (section
"Finite order pseudo-spectral solvers", the unit-pulse figure; "Conclusion": about 60
guard cells at p = 32), so each z subdomain, extended by enough guard cells on both sides,
can be advanced with its own Fourier transform of length N_local + 2 g and reproduce the
global update in its interior; with too few guard cells the periodic wrap of the local
transform leaves spurious fields.  This module builds that scheme from library handles:
one local handle of length N_local + 2 g (same Nr, Nm, order, time step and precision;
any length the library accepts, lengths that are not 7-smooth going through Bluestein rows)
is loaded with each subdomain's guarded window of E and B (pic_copy_window), its spectral
state is set from them (pic_fields_to_spectral), it advances one field step, and its
interior is written back into an output handle.

Only source-free field steps are decomposed: the global spectral current correction used
with sources (1/K^2 in z) is not local, and the paper only cites local variants of it.
All handles share one stream, so the copies are ordered with the steps.
"""
from __future__ import annotations

from . import binding as bd


class GuardedDomains:
    """n_domains equal z subdomains of a handle's grid, each advanced with `guard` cells
    of the neighbouring subdomains on both sides."""

    def __init__(self, cfg: bd.PicConfig, n_domains: int, guard: int, device="cuda:0", stream=None,
                 dht_path=None):
        if n_domains < 1 or cfg.Nz % n_domains:
            raise ValueError(f"Nz={cfg.Nz} is not a multiple of n_domains={n_domains}")
        self.n = n_domains
        self.L = cfg.Nz // n_domains
        self.g = int(guard)
        nz_loc = self.L + 2 * self.g
        if self.g < 0 or nz_loc > cfg.Nz:
            raise ValueError(f"local length {nz_loc} must be at most Nz={cfg.Nz}")
        lc = bd.make_config(nz_loc, cfg.Nr, cfg.Nm, cfg.dz, cfg.dr, cfg.dt, cfg.order_p, bool(cfg.filter),
                            cfg.precision, 0, cfg.q, cfg.mass)
        self.local = bd.Sim(lc, device=device, stream=stream)
        if dht_path is not None:   # FP64 form: the DHT path of the local handle (pic_set_dht_path)
            self.local.set_dht_path(dht_path)
        # source-free: zero deposit and previous spectral charge, kept zero by the steps
        self.local.set("DEP", self.local.zeros("DEP"))
        self.local.set("RHO_PREV_H", self.local.zeros("RHO_PREV_H"))

    def field_step(self, src: bd.Sim, out: bd.Sim):
        """out.E, out.B <- one source-free field step of src.E, src.B, subdomain by
        subdomain.  src and out may be the same handle only if src is not read again."""
        for d in range(self.n):
            z0 = d * self.L - self.g
            for name in ("E", "B"):
                src.copy_window_to(self.local, name, z0, self.L + 2 * self.g, 0)
            self.local.fields_to_spectral()
            self.local.field_step()
            for name in ("E", "B"):
                self.local.copy_window_to(out, name, self.g, self.L, d * self.L)

    def close(self):
        self.local.close()
