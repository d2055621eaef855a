"""Constants of the oracle (its own copy; nothing is shared with the CUDA side).

Physical constants are SI values.  The "stand-in" block holds the declared
constants of the waveform and precession stand-ins: the paper (Sec. II.A)
defers the IMRPhenomT coefficients and the NNLO Euler angles to earlier work,
so a model of the same structure is used instead.
"""
import math

# --- physical -----------------------------------------------------------
C_SI = 299792458.0                       # speed of light [m/s]
MTSUN_SI = 4.925490947641267e-06         # G M_sun / c^3 [s]
PC_SI = 3.085677581491367e16             # parsec [m]
GPC_S = 1.0e9 * PC_SI / C_SI             # one Gpc in light-seconds
AU_SI = 149597870700.0                   # astronomical unit [m]
AU_S = AU_SI / C_SI                      # AU in light-seconds
YEAR_SI = 31558149.763545603             # sidereal year [s]
OMEGA_ORB = 2.0 * math.pi / YEAR_SI      # guiding-centre angular rate [rad/s]

# --- LISA constellation (Sec. II.B) ------------------------------------
ARM_SI = 2.5e9                           # nominal arm length [m]
ARM_S = ARM_SI / C_SI                    # nominal light time [s]
# Keplerian model: first-order rigid triangle needs L = 2 sqrt(3) a e.
KEPLER_E0 = ARM_SI / (2.0 * math.sqrt(3.0) * AU_SI)
# per-spacecraft relative eccentricity offsets -> unequal, breathing arms
KEPLER_ETA = (0.0, 0.01, -0.01)

# --- Sangria analytic noise (Sec. II.B, PSD equations) -----------------
A_ACC = 2.4e-15                          # acceleration noise amplitude (a reading: the printed value is garbled)
A_OMS = 7.9e-12                          # optical metrology amplitude

# --- waveform stand-in (declared) --------------------------------------
F_MIN = 1.0e-4                           # start frequency of the (2,2) mode [Hz] (Table I)
T_TAPER = 1.0e4                          # Planck start-taper length [s]
F_HI_1 = 0.08                            # per-mode high-frequency taper start [Hz]
F_HI_2 = 0.09                            # per-mode high-frequency taper end [Hz]
X_MERGE = 2.0                            # x = nu (t_c - t)/(5M) where the ringdown attaches
C_SPIN = 0.5                             # spin-orbit coefficient of the frequency stand-in
# ringdown frequency ratio omega_lm / omega_22 and the mode list order
MODES = ((2, 2), (2, 1), (3, 3), (3, 2), (4, 4))
RD_RATIO = {(2, 2): 1.0, (2, 1): 0.75, (3, 3): 1.55, (3, 2): 1.25, (4, 4): 2.1}
