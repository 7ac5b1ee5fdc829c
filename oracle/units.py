"""Units and physical constants used by the oracle.

The paper writes Eq. 22 and Eq. 29 in Gaussian units and never states numeric
constants. Reading used throughout the oracle:

* lengths in Angstrom, wave numbers in 1/Angstrom, energies in kcal/mol;
* k_B = 0.0019872041 kcal/(mol K);
* the Coulomb constant q_a q_b / r -> COULOMB * q_a q_b / r with
  COULOMB = 332.0637 kcal Angstrom / (mol e^2);
* the unit "1" inside exp(-r) of Eq. 29 is 1/Angstrom and inside k^2 + 1 of
  Eq. 30 is 1/Angstrom^2.
"""
KB_KCAL = 0.0019872041          # kcal / (mol K)
COULOMB = 332.0637              # kcal Angstrom / (mol e^2)

# Singularity handling at r = 0 (the paper is silent): r^2 is floored at R2_FLOOR
# and the reduced potential beta*u is capped from above at BETA_U_CAP.
R2_FLOOR = 1.0e-8               # Angstrom^2
BETA_U_CAP = 1.0e4


def beta(temperature):
    """Inverse temperature 1/(k_B T) in mol/kcal."""
    return 1.0 / (KB_KCAL * temperature)
