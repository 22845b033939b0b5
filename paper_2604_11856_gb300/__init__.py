"""GB300-native hot path of RAPRAL (arXiv 2604.11856): line-by-line spectral
coefficients, ray march and wall radiative heat flux on one sm_103a GPU."""
